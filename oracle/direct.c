/* O(N^2) direct sum of Eq. (1.1), Sec. 1, in plain C and double precision.
 *
 *   p(x) = sum_y exp((i kappa - lambda) |x-y|) / (4 pi |x-y|^P) q(y),  skipping |x-y| <= eps
 *
 * (lambda = damping >= 0; 0 gives the paper's Helmholtz kernel; P = power, 1 or 2).
 *
 * Test infrastructure only: part of the CPU oracle, never linked into the
 * CUDA library.  X: nx*3 row-major, Y: ny*3 row-major, q: ny*nrhs complex
 * (interleaved re,im; column-major over right-hand sides), targets: nt
 * indices into X, out: nt*nrhs complex, column-major.
 */
#include <math.h>
#include <stdint.h>

void oracle_direct_sum(const double* X, int64_t nx, const double* Y, int64_t ny,
                       const double* q, int64_t nrhs, double kappa, double damping, double eps,
                       int power, const int64_t* targets, double* out, int64_t nt) {
    const double inv4pi = 1.0 / (4.0 * M_PI);
    (void)nx;
#pragma omp parallel for schedule(dynamic, 4)
    for (int64_t it = 0; it < nt; ++it) {
        const double* x = X + 3 * targets[it];
        for (int64_t r = 0; r < nrhs; ++r) {
            out[2 * (r * nt + it)] = 0.0;
            out[2 * (r * nt + it) + 1] = 0.0;
        }
        for (int64_t j = 0; j < ny; ++j) {
            double dx = x[0] - Y[3 * j], dy = x[1] - Y[3 * j + 1], dz = x[2] - Y[3 * j + 2];
            double rr = sqrt(dx * dx + dy * dy + dz * dz);
            if (!(rr > eps)) continue;
            double mag = exp(-damping * rr) * inv4pi / rr;
            if (power == 2) mag /= rr;
            double gr = cos(kappa * rr) * mag;
            double gi = sin(kappa * rr) * mag;
            for (int64_t r = 0; r < nrhs; ++r) {
                double qr = q[2 * (r * ny + j)], qi = q[2 * (r * ny + j) + 1];
                out[2 * (r * nt + it)] += gr * qr - gi * qi;
                out[2 * (r * nt + it) + 1] += gr * qi + gi * qr;
            }
        }
    }
}
