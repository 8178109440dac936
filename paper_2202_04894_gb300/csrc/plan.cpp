// Host-side plan construction (see plan.h).  Compiled with -ffp-contract=off
// so that every floating-point decision (Morton quantisation, MACs, regimes)
// is the plain IEEE result of the written expression.
#include "plan.h"
#include "symmetry.h"

#include <algorithm>
#include <cmath>
#include <cstdlib>
#include <exception>
#include <functional>
#include <numeric>
#include <stdexcept>
#include <thread>
#include <unordered_map>

namespace defmm {

// ---------------------------------------------------------------- levels / MAC
double Levels::side(int l) const { return side0 / (double)(1LL << l); }
double Levels::radius(int l) const { return std::sqrt(3.0) / 2 * side(l); }

// Strict MAC (footnote of Sec. 3.2) at low frequency, directional MAC
// max(kappa w^2, 2w) <= eta dist (Eq. macdirref, Sec. 4.2.2) at high frequency.
// The directional MAC reads A^2 <= F * S with S the integer squared gap.
void Levels::mac_terms(int l, double* A2, double* F) const {
    const double w = radius(l);
    const double A = std::max(kappa * w * w, 2 * w);
    const double s = side(l);
    *A2 = A * A;
    *F = eta * eta * s * s;
}

bool Levels::mac(int l, int64_t kx, int64_t ky, int64_t kz) const {
    int64_t ax = kx < 0 ? -kx : kx, ay = ky < 0 ? -ky : ky, az = kz < 0 ? -kz : kz;
    if (hf[l]) {
        int64_t gx = ax > 1 ? ax - 1 : 0, gy = ay > 1 ? ay - 1 : 0, gz = az > 1 ? az - 1 : 0;
        int64_t S = gx * gx + gy * gy + gz * gz;
        double A2, F;
        mac_terms(l, &A2, &F);
        return A2 <= F * (double)S;
    }
    return std::max(ax, std::max(ay, az)) >= 2;
}

// ---------------------------------------------------------------- directions
int64_t num_directions(int E) { return 6LL << (2 * E); }

static void direction_int(int E, int64_t d, int64_t w[3]) {
    int64_t n = 1LL << E;
    int64_t f = d / (n * n), rem = d % (n * n);
    int64_t i = rem / n, j = rem % n;
    int m = (int)(f / 2);
    int64_t sign = (f % 2 == 0) ? 1 : -1;
    int m1 = (m == 0) ? 1 : 0, m2 = (m == 2) ? 1 : 2;
    w[m] = sign * n;
    w[m1] = 2 * i + 1 - n;
    w[m2] = 2 * j + 1 - n;
}

void direction_vector(int E, int64_t d, double out[3]) {
    int64_t w[3];
    direction_int(E, d, w);
    double nrm = std::sqrt((double)(w[0] * w[0] + w[1] * w[1] + w[2] * w[2]));
    for (int a = 0; a < 3; ++a) out[a] = (double)w[a] / nrm;
}

int64_t direction_father(int E, int64_t d) {
    int64_t n = 1LL << E, h = n / 2;
    int64_t f = d / (n * n), rem = d % (n * n);
    int64_t i = rem / n, j = rem % n;
    return f * h * h + (i / 2) * h + (j / 2);
}

int64_t direction_negate(int E, int64_t d) {
    int64_t n = 1LL << E;
    int64_t f = d / (n * n), rem = d % (n * n);
    int64_t i = rem / n, j = rem % n;
    return (f ^ 1) * n * n + (n - 1 - i) * n + (n - 1 - j);
}

// argmax_v <v,k>/|v| over the level's directions, exact in integers; lowest
// index among ties for k whose first non-zero entry is positive, and the
// negated choice for the opposite k (so u(-k) = -u(k)).
static int64_t best_positive(int E, int64_t kx, int64_t ky, int64_t kz) {
    int64_t nd = num_directions(E);
    int64_t best = -1;
    __int128 bdot = 0, bn2 = 1;
    for (int64_t d = 0; d < nd; ++d) {
        int64_t w[3];
        direction_int(E, d, w);
        int64_t dot = w[0] * kx + w[1] * ky + w[2] * kz;
        if (dot <= 0) continue;
        int64_t n2 = w[0] * w[0] + w[1] * w[1] + w[2] * w[2];
        if (best < 0) {
            best = d; bdot = dot; bn2 = n2;
            continue;
        }
        __int128 lhs = (__int128)dot * dot * bn2;
        __int128 rhs = bdot * bdot * (__int128)n2;
        if (lhs > rhs) { best = d; bdot = dot; bn2 = n2; }
    }
    return best;
}

int64_t best_direction(int E, int64_t kx, int64_t ky, int64_t kz) {
    int64_t first = kx != 0 ? kx : (ky != 0 ? ky : kz);
    if (first > 0) return best_positive(E, kx, ky, kz);
    return direction_negate(E, best_positive(E, -kx, -ky, -kz));
}

// ---------------------------------------------------------------- symmetries
static const int kPerms[6][3] = DEFMM_PERM_TABLE;

Canon canonical(int64_t kx, int64_t ky, int64_t kz) {
    int64_t k[3] = {kx, ky, kz};
    const int64_t mag[3] = {kx < 0 ? -kx : kx, ky < 0 ? -ky : ky, kz < 0 ? -kz : kz};
    int order[3] = {0, 1, 2};
    // stable insertion sort of the axes by decreasing |k_i| (equal entries keep their order)
    for (int i = 1; i < 3; ++i)
        for (int j = i; j > 0 && mag[order[j - 1]] < mag[order[j]]; --j) std::swap(order[j - 1], order[j]);
    Canon c;
    for (int j = 0; j < 3; ++j) {
        int64_t v = k[order[j]];
        c.kbar[j] = (int)(v < 0 ? -v : v);
        c.sigma[order[j]] = j;
    }
    for (int i = 0; i < 3; ++i) c.sign[i] = k[i] < 0 ? -1 : 1;
    return c;
}

int transform_code(const Canon& c) {
    int pid = -1;
    for (int q = 0; q < 6; ++q)
        if (kPerms[q][0] == c.sigma[0] && kPerms[q][1] == c.sigma[1] && kPerms[q][2] == c.sigma[2])
            pid = q;
    int mask = (c.sign[0] < 0 ? 1 : 0) | (c.sign[1] < 0 ? 2 : 0) | (c.sign[2] < 0 ? 4 : 0);
    return pid * 8 + mask;
}

// ---------------------------------------------------------------- tree
static void build_tree(const double* P, int64_t n, const double corner[3], double side, int ncrit,
                       Tree& t) {
    std::vector<int64_t> key(n);
    const double scale = (double)(1LL << kMaxLevel);
    const int64_t gmax = (1LL << kMaxLevel) - 1;
    for (int64_t i = 0; i < n; ++i) {
        int64_t g[3];
        for (int a = 0; a < 3; ++a) {
            double v = (P[3 * i + a] - corner[a]) / side * scale;
            int64_t q = (int64_t)std::floor(v);
            g[a] = q < 0 ? 0 : (q > gmax ? gmax : q);
        }
        int64_t k = 0;
        for (int b = 0; b < kMaxLevel; ++b)
            for (int a = 0; a < 3; ++a) k |= ((g[a] >> b) & 1) << (3 * b + a);
        key[i] = k;
    }
    t.perm.resize(n);
    std::iota(t.perm.begin(), t.perm.end(), 0);
    std::stable_sort(t.perm.begin(), t.perm.end(), [&](int64_t a, int64_t b) { return key[a] < key[b]; });
    std::vector<int64_t> skey(n);
    for (int64_t i = 0; i < n; ++i) skey[i] = key[t.perm[i]];

    t.level = {0}; t.ix = {0}; t.iy = {0}; t.iz = {0};
    t.begin = {0}; t.end = {n}; t.parent = {-1};
    t.first_child.clear(); t.nchild.clear(); t.level_range.clear();
    int32_t start = 0;
    int lev = 0;
    while (start < (int32_t)t.level.size()) {
        int32_t stop = (int32_t)t.level.size();
        t.level_range.push_back({start, stop});
        for (int32_t c = start; c < stop; ++c) {
            int64_t b = t.begin[c], e = t.end[c];
            if (e - b > ncrit && lev < kMaxLevel) {
                int shift = 3 * (kMaxLevel - lev - 1);
                int64_t base = (skey[b] >> shift) >> 3 << 3;
                t.first_child.push_back((int32_t)t.level.size());
                int32_t nch = 0;
                int64_t lo = b;
                for (int o = 0; o < 8; ++o) {
                    // first index in [lo, e) whose prefix exceeds base + o
                    int64_t hi = std::upper_bound(skey.begin() + lo, skey.begin() + e, 0,
                                                  [&](int, int64_t kk) { return (kk >> shift) > base + o; }) -
                                 skey.begin();
                    if (hi > lo) {
                        t.level.push_back(lev + 1);
                        t.ix.push_back(2 * t.ix[c] + (o & 1));
                        t.iy.push_back(2 * t.iy[c] + ((o >> 1) & 1));
                        t.iz.push_back(2 * t.iz[c] + ((o >> 2) & 1));
                        t.begin.push_back(lo);
                        t.end.push_back(hi);
                        t.parent.push_back(c);
                        ++nch;
                    }
                    lo = hi;
                }
                t.nchild.push_back(nch);
            } else {
                t.first_child.push_back(-1);
                t.nchild.push_back(0);
            }
        }
        start = stop;
        ++lev;
    }
}

static int octant_of(const Tree& t, int32_t c) {
    return (t.ix[c] & 1) + 2 * (t.iy[c] & 1) + 4 * (t.iz[c] & 1);
}

static void sort_unique(std::vector<int32_t>& v) {
    std::sort(v.begin(), v.end());
    v.erase(std::unique(v.begin(), v.end()), v.end());
}

// Alg. 1 from (root, root), breadth first: the pairs of one level in order,
// each giving an M2L pair (with its best direction), a P2P pair or its son
// pairs in (a, b) order for the next level; then the marks of Alg. 2 (the
// directions of each cell's M2L pairs).
static void dual_tree_traversal(HostPlan& hp) {
    const Tree& tt = hp.tt;
    const Tree& ts = hp.ts();
    const Levels& lv = hp.lv;
    std::unordered_map<int64_t, int32_t> dir_memo;
    auto pair_dir = [&](int l, int64_t kx, int64_t ky, int64_t kz) -> int32_t {
        if (!lv.hf[l]) return -1;
        int64_t key = ((((int64_t)l * 4096 + (kx + 2048)) * 4096) + (ky + 2048)) * 4096 + (kz + 2048);
        auto it = dir_memo.find(key);
        if (it != dir_memo.end()) return it->second;
        int32_t u = (int32_t)best_direction(lv.E(l), kx, ky, kz);
        dir_memo[key] = u;
        return u;
    };
    std::vector<std::array<int32_t, 2>> cur = {{0, 0}}, next;
    while (!cur.empty()) {
        next.clear();
        for (const auto& pr : cur) {
            const int32_t t = pr[0], s = pr[1];
            const int l = tt.level[t];
            const int64_t kx = (int64_t)tt.ix[t] - ts.ix[s], ky = (int64_t)tt.iy[t] - ts.iy[s],
                          kz = (int64_t)tt.iz[t] - ts.iz[s];
            if (lv.mac(l, kx, ky, kz)) {
                hp.m2l.push_back({t, s, pair_dir(l, kx, ky, kz)});
            } else if (tt.leaf(t) || ts.leaf(s)) {
                hp.p2p.push_back({t, s});
            } else {
                for (int32_t a = 0; a < tt.nchild[t]; ++a)
                    for (int32_t b = 0; b < ts.nchild[s]; ++b)
                        next.push_back({tt.first_child[t] + a, ts.first_child[s] + b});
            }
        }
        cur.swap(next);
    }
    hp.marks_t.assign(tt.ncell(), {});
    hp.marks_s.assign(ts.ncell(), {});
    for (auto& pr : hp.m2l)
        if (pr[2] >= 0) {
            hp.marks_t[pr[0]].push_back(pr[2]);
            hp.marks_s[pr[1]].push_back(pr[2]);
        }
}

// Threads for the plan's parallel passes: up to 16 (hardware permitting), or
// DEFMM_PLAN_THREADS (1..16).
static int plan_threads() {
    int n = (int)std::min<unsigned>(16u, std::max(1u, std::thread::hardware_concurrency()));
    if (const char* env = std::getenv("DEFMM_PLAN_THREADS")) {
        const int v = std::atoi(env);
        if (v >= 1) n = std::min(v, 16);
    }
    return n;
}

// fn(begin, end) over nthreads equal slices of [0, n); slices whose thread cannot
// be created run on this thread; an exception in any slice is rethrown here.
static void parallel_slices(size_t n, int nthreads, const std::function<void(size_t, size_t)>& fn) {
    nthreads = std::max(1, std::min<int>(nthreads, (int)std::max<size_t>(1, n)));
    std::vector<std::exception_ptr> failed(nthreads);
    auto run = [&](int j) {
        try {
            fn(n * j / nthreads, n * (j + 1) / nthreads);
        } catch (...) {
            failed[j] = std::current_exception();
        }
    };
    std::vector<std::thread> pool;
    int started = 1;
    try {
        for (; started < nthreads; ++started) pool.emplace_back(run, started);
    } catch (...) {
    }
    run(0);
    for (int j = started; j < nthreads; ++j) run(j);
    for (auto& th : pool) th.join();
    for (auto& e : failed)
        if (e) std::rethrow_exception(e);
}

// ---------------------------------------------------------------- plan
template <typename U> static bool units_for_leaf_empty(const std::vector<U>& units, int32_t li) {
    return units.empty() || units.back().leaf != li;
}

void build_host_plan(const double* X, int64_t nx, const double* Y, int64_t ny, double kappa,
                     int order, int leaf, double eta, double hf_kw, int fft_n, double self_eps,
                     int chunk_blocks, HostPlan& hp, const FrontEnd* front) {
    if (nx < 1 || ny < 1) throw std::runtime_error("nx and ny must be >= 1");
    if (order < 2 || order > kMaxOrder) throw std::runtime_error("order must be in [2, 8]");
    if (leaf < 1) throw std::runtime_error("leaf_size must be >= 1");
    if (!(kappa >= 0) || !std::isfinite(kappa)) throw std::runtime_error("kappa must be finite and >= 0");
    if (!(eta > 0)) throw std::runtime_error("eta must be > 0");
    if (nx > (1LL << 31) - 2 || ny > (1LL << 31) - 2) throw std::runtime_error("too many points (> 2^31)");
    hp.nx = nx; hp.ny = ny; hp.same = (Y == nullptr);
    hp.kappa = kappa; hp.p = order; hp.eta = eta; hp.hf_kw = hf_kw; hp.self_eps_rel = self_eps;
    hp.N = fft_n > 0 ? fft_n : 2 * order - 1;
    if (hp.N < 2 * order - 1) throw std::runtime_error("fft_n must be >= 2*order - 1");
    if (hp.N > 16) throw std::runtime_error("fft_n must be <= 16");
    hp.NF = hp.N * hp.N * hp.N;
    hp.NFpad = (hp.NF + 3) / 4 * 4;
    hp.P3 = order * order * order;
    for (int64_t i = 0; i < 3 * nx; ++i)
        if (!std::isfinite(X[i])) throw std::runtime_error("non-finite target coordinate");
    if (Y)
        for (int64_t i = 0; i < 3 * ny; ++i)
            if (!std::isfinite(Y[i])) throw std::runtime_error("non-finite source coordinate");

    // bounding cube of X u Y, enlarged by 1 + 2^-20 (Sec. 1, Sec. 2.3)
    double lo[3], hi[3];
    for (int a = 0; a < 3; ++a) { lo[a] = X[a]; hi[a] = X[a]; }
    auto grow = [&](const double* P, int64_t n) {
        for (int64_t i = 0; i < n; ++i)
            for (int a = 0; a < 3; ++a) {
                lo[a] = std::min(lo[a], P[3 * i + a]);
                hi[a] = std::max(hi[a], P[3 * i + a]);
            }
    };
    grow(X, nx);
    if (Y) grow(Y, ny);
    double d = std::max(hi[0] - lo[0], std::max(hi[1] - lo[1], hi[2] - lo[2]));
    if (d == 0.0) d = 1.0;
    hp.d_aabb = d;
    hp.side = d * (1.0 + std::ldexp(1.0, -20));
    for (int a = 0; a < 3; ++a) hp.corner[a] = (lo[a] + hi[a]) / 2.0 - hp.side / 2.0;
    hp.eps_self = self_eps * d;


    Levels& lv = hp.lv;
    lv.side0 = hp.side; lv.kappa = kappa; lv.eta = eta; lv.hf_kw = hf_kw;
    lv.l_hf = -1;
    for (int l = 0; l < kNumLevels; ++l) {
        lv.hf[l] = kappa * lv.radius(l) > hf_kw;
        if (lv.hf[l]) lv.l_hf = l;
    }
    lv.hf[kNumLevels] = false;
    if (lv.l_hf >= 0 && lv.l_hf > 12)
        throw std::runtime_error("kappa*D too large: more than 12 high-frequency levels");

    if (front) {
        (*front)(hp);   // trees, traversal, directions and Alg. 2 marks built elsewhere (the device)
    } else {
        build_tree(X, nx, hp.corner, hp.side, leaf, hp.tt);
        if (Y) build_tree(Y, ny, hp.corner, hp.side, leaf, hp.ts_own);
        dual_tree_traversal(hp);
    }
    const Tree& tt = hp.tt;
    const Tree& ts = hp.ts();

    // ---- Alg. 3 blank downward pass on both trees (the marks of Alg. 2 are in place)
    // Cells are stored level by level; a level's cells are independent (each writes
    // its own marks and those of its sons), so a level's cells run on several threads.
    auto downward = [&](const Tree& tr, std::vector<std::vector<int32_t>>& marks) {
        auto cell = [&](int32_t c) {
            int l = tr.level[c];
            if (!lv.hf[l]) {
                marks[c].assign(1, -1);
                return;
            }
            sort_unique(marks[c]);
            if (!lv.hf[l + 1]) return;
            for (int32_t a = 0; a < tr.nchild[c]; ++a)
                for (int32_t u : marks[c])
                    marks[tr.first_child[c] + a].push_back((int32_t)direction_father(lv.E(l), u));
        };
        for (const auto& lr : tr.level_range) {
            const size_t n = (size_t)(lr.second - lr.first);
            parallel_slices(n, n >= 4096 ? plan_threads() : 1, [&](size_t i0, size_t i1) {
                for (size_t i = i0; i < i1; ++i) cell(lr.first + (int32_t)i);
            });
        }
    };
    downward(tt, hp.marks_t);
    downward(ts, hp.marks_s);

    // ---- effective expansions
    auto enumerate = [&](const Tree& tr, const std::vector<std::vector<int32_t>>& marks,
                         std::vector<int32_t>& cell, std::vector<int32_t>& dir,
                         std::vector<int32_t>& first, std::vector<int32_t>& count) {
        first.assign(tr.ncell(), 0);
        count.assign(tr.ncell(), 0);
        for (int32_t c = 0; c < tr.ncell(); ++c) {
            first[c] = (int32_t)cell.size();
            for (int32_t u : marks[c]) { cell.push_back(c); dir.push_back(u); }
            count[c] = (int32_t)marks[c].size();
        }
    };
    enumerate(ts, hp.marks_s, hp.m_cell, hp.m_dir, hp.m_first, hp.m_count);
    enumerate(tt, hp.marks_t, hp.l_cell, hp.l_dir, hp.l_first, hp.l_count);
    auto find_exp = [](const std::vector<int32_t>& dir, int32_t first, int32_t count, int32_t u) -> int32_t {
        auto b = dir.begin() + first, e = b + count;
        auto it = std::lower_bound(b, e, u);
        if (it == e || *it != u) return -1;
        return (int32_t)(it - dir.begin());
    };

    // ---- phase slots per (level, direction) (Sec. 5.2.1 diagonal factors)
    std::unordered_map<int64_t, int32_t> slot_of;
    const int p = order;
    auto get_slot = [&](int l, int32_t u) -> int32_t {
        if (u < 0) return -1;
        int64_t key = (int64_t)l * (1LL << 40) + u;
        auto it = slot_of.find(key);
        if (it != slot_of.end()) return it->second;
        int32_t s = (int32_t)hp.slot_level.size();
        slot_of[key] = s;
        hp.slot_level.push_back(l);
        hp.slot_dir.push_back(u);
        double v[3];
        direction_vector(lv.E(l), u, v);
        for (int a = 0; a < 3; ++a) hp.slot_u.push_back(v[a]);
        double side = lv.side(l);
        for (int a = 0; a < 3; ++a)
            for (int m = 0; m < p; ++m) {
                double arg = kappa * side * ((double)m / (p - 1) - 0.5) * v[a];
                hp.slot_P.push_back(std::cos(arg));
                hp.slot_P.push_back(std::sin(arg));
            }
        for (int a = 0; a < 3; ++a)
            for (int o = 0; o < 2; ++o)
                for (int b = 0; b < p; ++b) {
                    double arg = kappa * side * ((o + (double)b / (p - 1)) / 2 - 0.5) * v[a];
                    hp.slot_Q.push_back(std::cos(arg));
                    hp.slot_Q.push_back(std::sin(arg));
                }
        return s;
    };
    hp.m_slot.resize(hp.m_cell.size());
    for (size_t e = 0; e < hp.m_cell.size(); ++e) hp.m_slot[e] = get_slot(ts.level[hp.m_cell[e]], hp.m_dir[e]);
    hp.l_slot.resize(hp.l_cell.size());
    for (size_t e = 0; e < hp.l_cell.size(); ++e) hp.l_slot[e] = get_slot(tt.level[hp.l_cell[e]], hp.l_dir[e]);

    // 1-D interpolation matrices M1[o][a][b] = l_a((o + b/(p-1))/2) and twiddles
    hp.m1.assign(2 * p * p, 0.0);
    for (int o = 0; o < 2; ++o)
        for (int a = 0; a < p; ++a)
            for (int b = 0; b < p; ++b) {
                double t = (o + (double)b / (p - 1)) / 2;
                double v = 1.0;
                for (int m = 0; m < p; ++m)
                    if (m != a) v *= (t - (double)m / (p - 1)) / ((double)a / (p - 1) - (double)m / (p - 1));
                hp.m1[(o * p + a) * p + b] = v;
            }
    hp.tw.assign(2 * hp.N, 0.0);
    for (int m = 0; m < hp.N; ++m) {
        double ang = 2.0 * 3.14159265358979323846 * m / hp.N;
        hp.tw[2 * m] = std::cos(ang);
        hp.tw[2 * m + 1] = std::sin(ang);
    }

    // ---- spectra and M2L tables
    std::unordered_map<int64_t, int32_t> spec_of;
    struct PairRec { int32_t tgt, src, spec, code, order; };
    std::vector<PairRec> recs;
    recs.reserve(hp.m2l.size());
    std::vector<int32_t> is_src(hp.m_cell.size(), 0);
    // spectrum and transform code of an offset: found once per (level, offset)
    // and kept in a dense per-level table while that stays small
    auto spectrum_of = [&](int l, int64_t kx, int64_t ky, int64_t kz, int32_t* code) {
        const Canon cn = canonical(kx, ky, kz);
        const int64_t key = (((int64_t)l * 4096 + cn.kbar[0]) * 4096 + cn.kbar[1]) * 4096 + cn.kbar[2];
        *code = transform_code(cn);
        auto it = spec_of.find(key);
        if (it != spec_of.end()) return it->second;
        const int32_t sid = (int32_t)hp.spec_level.size();
        spec_of[key] = sid;
        hp.spec_level.push_back(l);
        hp.spec_kbar.push_back({cn.kbar[0], cn.kbar[1], cn.kbar[2]});
        return sid;
    };
    // the target and source expansion of every pair and the largest offset per level
    // (independent per pair: slices on several threads, one maximum per slice), then
    // the spectra in the order the pairs first use them (one pass)
    std::vector<int64_t> kmax(kNumLevels + 1, -1);
    recs.resize(hp.m2l.size());
    {
        const int nth = hp.m2l.size() >= ((size_t)1 << 20) ? plan_threads() : 1;
        std::vector<std::vector<int64_t>> kmax_of(nth, std::vector<int64_t>(kNumLevels + 1, -1));
        parallel_slices((size_t)nth, nth, [&](size_t j0, size_t j1) {
            for (size_t j = j0; j < j1; ++j) {
                std::vector<int64_t>& km = kmax_of[j];
                const size_t i0 = hp.m2l.size() * j / nth, i1 = hp.m2l.size() * (j + 1) / nth;
                for (size_t i = i0; i < i1; ++i) {
                    const auto& pr = hp.m2l[i];
                    const int32_t te = find_exp(hp.l_dir, hp.l_first[pr[0]], hp.l_count[pr[0]], pr[2]);
                    const int32_t se = find_exp(hp.m_dir, hp.m_first[pr[1]], hp.m_count[pr[1]], pr[2]);
                    recs[i] = {te, se, 0, 0, (int32_t)i};
                    const int l = tt.level[pr[0]];
                    const int64_t k = std::max({std::llabs((int64_t)tt.ix[pr[0]] - ts.ix[pr[1]]),
                                                std::llabs((int64_t)tt.iy[pr[0]] - ts.iy[pr[1]]),
                                                std::llabs((int64_t)tt.iz[pr[0]] - ts.iz[pr[1]])});
                    km[l] = std::max(km[l], k);
                }
            }
        });
        for (const auto& km : kmax_of)
            for (int l = 0; l <= kNumLevels; ++l) kmax[l] = std::max(kmax[l], km[l]);
    }
    // one dense table per level from offset to (spectrum, code), concatenated, while it stays small
    std::vector<int64_t> tbase(kNumLevels + 2, 0);
    for (int l = 0; l <= kNumLevels; ++l) {
        const int64_t w = 2 * kmax[l] + 1;
        const bool dense = kmax[l] >= 0 && w * w * w <= (int64_t(1) << 22);
        tbase[l + 1] = tbase[l] + (dense ? w * w * w : 0);
    }
    std::vector<int32_t> by_offset((size_t)tbase[kNumLevels + 1], -1);   // sid * 64 + code, -1: not yet seen
    auto offset_of = [&](size_t i, int* l, int64_t* kx, int64_t* ky, int64_t* kz) {
        const int32_t t = hp.m2l[i][0], s = hp.m2l[i][1];
        *l = tt.level[t];
        *kx = (int64_t)tt.ix[t] - ts.ix[s];
        *ky = (int64_t)tt.iy[t] - ts.iy[s];
        *kz = (int64_t)tt.iz[t] - ts.iz[s];
    };
    // each pair's table slot (independent per pair; -1 where its level has no table), kept in
    // recs[i].spec until the spectra are numbered in the order the pairs first use them
    parallel_slices(hp.m2l.size(), hp.m2l.size() >= ((size_t)1 << 20) ? plan_threads() : 1,
                    [&](size_t i0, size_t i1) {
        for (size_t i = i0; i < i1; ++i) {
            int l;
            int64_t kx, ky, kz;
            offset_of(i, &l, &kx, &ky, &kz);
            const int64_t K = kmax[l], w = 2 * K + 1;
            recs[i].spec = tbase[l + 1] > tbase[l] ? (int32_t)(tbase[l] + ((kx + K) * w + (ky + K)) * w + (kz + K)) : -1;
        }
    });
    for (size_t i = 0; i < hp.m2l.size(); ++i) {
        PairRec& r = recs[i];
        if (r.tgt < 0 || r.src < 0) throw std::runtime_error("internal: M2L expansion missing");
        int32_t sid, code;
        if (r.spec >= 0) {
            int32_t& v = by_offset[(size_t)r.spec];
            if (v < 0) {
                int l;
                int64_t kx, ky, kz;
                offset_of(i, &l, &kx, &ky, &kz);
                sid = spectrum_of(l, kx, ky, kz, &code);
                v = sid * 64 + code;
            }
            sid = v >> 6;
            code = v & 63;
        } else {
            int l;
            int64_t kx, ky, kz;
            offset_of(i, &l, &kx, &ky, &kz);
            sid = spectrum_of(l, kx, ky, kz, &code);
        }
        r.spec = sid;
        r.code = code;
        is_src[r.src] = 1;
    }
    hp.mhat_of_m.assign(hp.m_cell.size(), -1);
    for (size_t e = 0; e < hp.m_cell.size(); ++e)
        if (is_src[e]) {
            hp.mhat_of_m[e] = (int32_t)hp.m2f_list.size();
            hp.m2f_list.push_back((int32_t)e);
        }
    // ---- M2L groups and chunks (sibling targets sharing a father and a direction)
    {
        // blocks per chunk: about 35 KB of complex64 for N <= 8 (13 blocks for N = 7:
        // two stages of the row kernel still fit three blocks of 7 members per SM, and
        // each staged block serves more pairs; measured against 8 to 24 blocks on the
        // 10^6-point sphere, cube and ellipsoid); for longer DFTs up to 8, as long as
        // two stages of complex128 fit in shared memory
        int max_blocks = hp.N <= 8 ? std::max(2, std::min(31, 35840 / (hp.NFpad * 8)))
                                   : std::max(2, std::min(8, 115200 / (hp.NFpad * 16)));
        if (chunk_blocks > 0) max_blocks = std::max(2, std::min(max_blocks, chunk_blocks));   // may only shrink
        hp.chk_max_blocks = max_blocks;
        // groups of at most 4 siblings run in blocks of 4 members, five per SM: their
        // chunks keep about 22 KB (8 blocks for N = 7) so that two stages still fit
        const int max_blocks_small = hp.N <= 8 ? std::min(max_blocks, std::max(2, std::min(31, 22528 / (hp.NFpad * 8))))
                                               : max_blocks;
        struct Op { int32_t member, src_parent, src, spec, code; };
        std::unordered_map<int64_t, int32_t> group_of;   // (father cell, direction) -> group
        std::vector<std::vector<int32_t>> members;        // local expansion ids
        // group and member slot of each target expansion, in increasing target
        // expansion order (groups and members numbered in that order)
        std::vector<int32_t> grp_of_te(hp.l_cell.size(), -1), slot_of_te(hp.l_cell.size(), -1);
        std::vector<int64_t> tcount(hp.l_cell.size(), 0), gcount;
        for (const PairRec& r : recs) ++tcount[r.tgt];
        for (size_t te = 0; te < hp.l_cell.size(); ++te) {
            if (tcount[te] == 0) continue;
            const int32_t t = hp.l_cell[te], u = hp.l_dir[te];
            const int64_t key = (int64_t)tt.parent[t] * (1LL << 32) + (int64_t)(u + 1);
            auto it = group_of.find(key);
            int32_t g;
            if (it == group_of.end()) {
                g = (int32_t)members.size();
                group_of[key] = g;
                members.push_back({});
                gcount.push_back(0);
            } else {
                g = it->second;
            }
            if (members[g].size() >= 8) throw std::runtime_error("internal: more than 8 siblings in an M2L group");
            grp_of_te[te] = g;
            slot_of_te[te] = (int32_t)members[g].size();
            members[g].push_back((int32_t)te);
            gcount[g] += tcount[te];
        }
        // every group's ops in one array (CSR; their order within a group does not
        // matter: each group's ops are sorted by a unique key below)
        std::vector<int64_t> gop_off(members.size() + 1, 0);
        for (size_t g = 0; g < members.size(); ++g) gop_off[g + 1] = gop_off[g] + gcount[g];
        std::vector<Op> gop_all(recs.size());
        {
            std::vector<int64_t> at(gop_off.begin(), gop_off.end() - 1);
            for (size_t i = 0; i < recs.size(); ++i) {
                const int32_t te = recs[i].tgt, s_cell = hp.m_cell[recs[i].src];
                gop_all[(size_t)at[grp_of_te[te]]++] = {slot_of_te[te], ts.parent[s_cell], hp.mhat_of_m[recs[i].src],
                                                        recs[i].spec, recs[i].code};
            }
        }
        auto gops_size = [&](int32_t g) { return gop_off[g + 1] - gop_off[g]; };
        // heaviest groups first
        std::vector<int32_t> gorder(members.size());
        std::iota(gorder.begin(), gorder.end(), 0);
        std::stable_sort(gorder.begin(), gorder.end(), [&](int32_t a, int32_t b) { return gops_size(a) > gops_size(b); });
        // Chunks of each group, built by several threads over contiguous slices of
        // the group order into their own arrays (block and op offsets relative to
        // the slice), then concatenated in order: the same tables as one pass.
        struct Slice {
            std::vector<int32_t> members, member_n, chunk_n;           // per group
            std::vector<int32_t> nspec, blk, blk_end, op, op_off;      // per chunk (ends relative)
            int32_t stage[3] = {0, 0, 0};
        };
        auto build_slice = [&](size_t q0, size_t q1, Slice& out) {
            std::vector<int32_t> specs, srcs;   // a chunk's distinct blocks, in first-use order
            struct ChunkOp { int32_t member, code, sb, mb; };   // an op with its block positions
            std::vector<ChunkOp> chunk, by_member;
            for (size_t q = q0; q < q1; ++q) {
                const int32_t g = gorder[q];
                const int budget = members[g].size() <= 4 ? max_blocks_small : max_blocks;
                out.members.insert(out.members.end(), members[g].begin(), members[g].end());
                out.member_n.push_back((int32_t)members[g].size());
                Op* const ops_b = gop_all.data() + gop_off[g];
                Op* const ops_e = gop_all.data() + gop_off[g + 1];
                // sources grouped by their father: a chunk then covers about one father's sons
                std::stable_sort(ops_b, ops_e, [](const Op& a, const Op& b) {
                    if (a.src_parent != b.src_parent) return a.src_parent < b.src_parent;
                    if (a.src != b.src) return a.src < b.src;
                    return a.member < b.member;
                });
                int32_t nchunk = 0;
                size_t i = 0;
                const size_t nops = (size_t)(ops_e - ops_b);
                while (i < nops) {
                    specs.clear();
                    srcs.clear();
                    chunk.clear();
                    while (i < nops) {
                        const Op& o = ops_b[i];
                        const auto sp = std::find(specs.begin(), specs.end(), o.spec);
                        const bool new_sp = sp == specs.end();
                        // ops are sorted by (source father, source) and a source has one
                        // father, so each source's ops form one run
                        const bool new_src = srcs.empty() || srcs.back() != o.src;
                        const int need = (int)specs.size() + (int)srcs.size() + (new_sp ? 1 : 0) + (new_src ? 1 : 0);
                        if (!chunk.empty() && need > budget) break;
                        const int32_t sb = (int32_t)(sp - specs.begin());
                        if (new_sp) specs.push_back(o.spec);
                        if (new_src) srcs.push_back(o.src);
                        chunk.push_back({o.member, o.code, sb, (int32_t)srcs.size() - 1});
                        ++i;
                    }
                    const int32_t nsp = (int32_t)specs.size();
                    for (int v = 0; v < 3; ++v)   // stage size when 1, 2, 4 right-hand sides share it
                        out.stage[v] = std::max(out.stage[v], nsp + (1 << v) * (int32_t)srcs.size());
                    out.nspec.push_back(nsp);
                    out.blk.insert(out.blk.end(), specs.begin(), specs.end());
                    out.blk.insert(out.blk.end(), srcs.begin(), srcs.end());
                    out.blk_end.push_back((int32_t)out.blk.size());
                    // ops by member, in chunk order within a member (a stable bucket sort)
                    int32_t at[9] = {0, 0, 0, 0, 0, 0, 0, 0, 0};
                    for (const ChunkOp& o : chunk) ++at[o.member + 1];
                    for (int m = 0; m < 8; ++m) at[m + 1] += at[m];
                    by_member.resize(chunk.size());
                    for (const ChunkOp& o : chunk) by_member[at[o.member]++] = o;
                    const int32_t base = (int32_t)out.op.size();
                    size_t k = 0;
                    for (int m = 0; m < 8; ++m) {
                        out.op_off.push_back(base + (int32_t)k);
                        while (k < by_member.size() && by_member[k].member == m) {
                            const ChunkOp& o = by_member[k];
                            out.op.push_back(o.sb | ((nsp + o.mb) << 8) | (o.code << 16));
                            ++k;
                        }
                    }
                    out.op_off.push_back(base + (int32_t)k);
                    ++nchunk;
                }
                out.chunk_n.push_back(nchunk);
            }
        };
        // slices of about equal op counts; one thread for small plans
        const size_t ng = gorder.size();
        // an explicit DEFMM_PLAN_THREADS applies to any plan size (tests compare counts)
        int nthreads = plan_threads();
        if (recs.size() < (size_t)1 << 20 && !std::getenv("DEFMM_PLAN_THREADS")) nthreads = 1;
        std::vector<size_t> cut(1, 0);
        {
            size_t acc = 0, k = 1;
            for (size_t q = 0; q < ng && (int)k < nthreads; ++q) {
                acc += (size_t)gops_size(gorder[q]);
                if (acc * nthreads >= recs.size() * k) { cut.push_back(q + 1); ++k; }
            }
            cut.push_back(ng);
        }
        std::vector<Slice> slices(cut.size() - 1);
        {
            std::vector<std::exception_ptr> failed(slices.size());
            auto run = [&](size_t j) {   // an exception (allocation) is carried back to this thread
                try {
                    build_slice(cut[j], cut[j + 1], slices[j]);
                } catch (...) {
                    failed[j] = std::current_exception();
                }
            };
            // slices whose thread cannot be created run here, after slice 0
            std::vector<std::thread> pool;
            size_t started = 1;
            try {
                for (; started < slices.size(); ++started) pool.emplace_back(run, started);
            } catch (...) {
            }
            run(0);
            for (size_t j = started; j < slices.size(); ++j) run(j);
            for (auto& th : pool) th.join();
            for (auto& e : failed)
                if (e) std::rethrow_exception(e);
        }
        // concatenation: every slice's part of each table at its prefix offsets, copied in parallel
        struct Base { size_t grp, mem, chk, blk, op; };
        std::vector<Base> base(slices.size() + 1, Base{0, 0, 0, 0, 0});
        for (size_t j = 0; j < slices.size(); ++j) {
            const Slice& sl = slices[j];
            base[j + 1] = {base[j].grp + sl.member_n.size(), base[j].mem + sl.members.size(),
                           base[j].chk + sl.nspec.size(), base[j].blk + sl.blk.size(), base[j].op + sl.op.size()};
            for (int v = 0; v < 3; ++v) hp.chk_stage_blocks[v] = std::max(hp.chk_stage_blocks[v], sl.stage[v]);
        }
        const Base& all = base.back();
        if (all.op > (size_t)INT32_MAX || all.blk > (size_t)INT32_MAX) throw std::runtime_error("M2L schedule too large");
        hp.grp_members.resize(all.mem);
        hp.grp_member_off.assign(all.grp + 1, 0);
        hp.grp_chunk_off.assign(all.grp + 1, 0);
        hp.chk_nspec.resize(all.chk);
        hp.chk_blk.resize(all.blk);
        hp.chk_blk_off.assign(all.chk + 1, 0);
        hp.chk_op.resize(all.op);
        hp.chk_op_off.resize(9 * all.chk);
        parallel_slices(slices.size(), (int)slices.size(), [&](size_t j0, size_t j1) {
            for (size_t j = j0; j < j1; ++j) {
                const Slice& sl = slices[j];
                const Base& b = base[j];
                std::copy(sl.members.begin(), sl.members.end(), hp.grp_members.begin() + b.mem);
                int32_t m = (int32_t)b.mem, ck = (int32_t)b.chk;
                for (size_t i = 0; i < sl.member_n.size(); ++i) {
                    m += sl.member_n[i];
                    ck += sl.chunk_n[i];
                    hp.grp_member_off[b.grp + i + 1] = m;
                    hp.grp_chunk_off[b.grp + i + 1] = ck;
                }
                std::copy(sl.nspec.begin(), sl.nspec.end(), hp.chk_nspec.begin() + b.chk);
                std::copy(sl.blk.begin(), sl.blk.end(), hp.chk_blk.begin() + b.blk);
                for (size_t i = 0; i < sl.blk_end.size(); ++i) hp.chk_blk_off[b.chk + i + 1] = (int32_t)b.blk + sl.blk_end[i];
                std::copy(sl.op.begin(), sl.op.end(), hp.chk_op.begin() + b.op);
                for (size_t i = 0; i < sl.op_off.size(); ++i) hp.chk_op_off[9 * b.chk + i] = (int32_t)b.op + sl.op_off[i];
            }
        });
        // the same groups cut into blocks of at most 4 members (heaviest first)
        for (size_t gi = 0; gi + 1 < hp.grp_member_off.size(); ++gi) {
            const int nm = hp.grp_member_off[gi + 1] - hp.grp_member_off[gi];
            for (int h = 0; 4 * h < nm; ++h) hp.grp_half.push_back((int32_t)(2 * gi + h));
        }
    }

    // ---- M2M per parent level (source tree)
    int nlev_s = (int)ts.level_range.size();
    hp.m2m_lvl.assign(nlev_s, {});
    for (int l = 0; l < nlev_s; ++l) {
        for (int32_t c = ts.level_range[l].first; c < ts.level_range[l].second; ++c) {
            if (ts.leaf(c) || hp.m_count[c] == 0) continue;
            for (int32_t e = hp.m_first[c]; e < hp.m_first[c] + hp.m_count[c]; ++e) {
                int32_t v = hp.m_dir[e];
                int32_t u2 = (v < 0 || !lv.hf[l + 1]) ? -1 : (int32_t)direction_father(lv.E(l), v);
                int32_t ch[8] = {-1, -1, -1, -1, -1, -1, -1, -1};
                for (int32_t a = 0; a < ts.nchild[c]; ++a) {
                    int32_t c2 = ts.first_child[c] + a;
                    int32_t ce = find_exp(hp.m_dir, hp.m_first[c2], hp.m_count[c2], u2);
                    if (ce < 0) throw std::runtime_error("internal: M2M child expansion missing");
                    ch[octant_of(ts, c2)] = ce;
                }
                hp.m2m_lvl[l].push_back(e);
                for (int o = 0; o < 8; ++o) hp.m2m_lvl[l].push_back(ch[o]);
            }
        }
    }

    // ---- L2L per child level (target tree)
    int nlev_t = (int)tt.level_range.size();
    hp.l2l_lvl.assign(nlev_t, {});
    hp.l2l_par.assign(nlev_t, {});
    for (int l = 1; l < nlev_t; ++l) {
        for (int32_t c = tt.level_range[l].first; c < tt.level_range[l].second; ++c) {
            int32_t par = tt.parent[c];
            if (hp.l_count[par] == 0) continue;
            for (int32_t e = hp.l_first[c]; e < hp.l_first[c] + hp.l_count[c]; ++e) {
                int32_t u = hp.l_dir[e];
                int32_t first = (int32_t)hp.l2l_par[l].size();
                for (int32_t pe = hp.l_first[par]; pe < hp.l_first[par] + hp.l_count[par]; ++pe) {
                    int32_t v = hp.l_dir[pe];
                    int32_t want = (v < 0 || !lv.hf[l]) ? -1 : (int32_t)direction_father(lv.E(l - 1), v);
                    if (want == u) hp.l2l_par[l].push_back(pe);
                }
                int32_t cnt = (int32_t)hp.l2l_par[l].size() - first;
                if (cnt == 0) continue;
                hp.l2l_lvl[l].push_back(e);
                hp.l2l_lvl[l].push_back(octant_of(tt, c));
                hp.l2l_lvl[l].push_back(first);
                hp.l2l_lvl[l].push_back(cnt);
            }
        }
    }

    // ---- leaves for P2M / L2P
    for (int32_t c = 0; c < ts.ncell(); ++c)
        if (ts.leaf(c) && hp.m_count[c] > 0) hp.p2m_cells.push_back(c);
    for (int32_t c = 0; c < tt.ncell(); ++c)
        if (tt.leaf(c) && hp.l_count[c] > 0) hp.l2p_cells.push_back(c);

    // ---- P2P: per target leaf, the source ranges of its near pairs
    // each near pair's source cell to every target leaf under its target cell (the
    // order within a leaf does not matter: a leaf's list is sorted below)
    std::vector<std::vector<int32_t>> near(tt.ncell());
    {
        std::vector<int32_t> stack;
        for (const auto& pr : hp.p2p) {
            if (tt.leaf(pr[0])) { near[pr[0]].push_back(pr[1]); continue; }
            stack.assign(1, pr[0]);
            while (!stack.empty()) {
                const int32_t t = stack.back();
                stack.pop_back();
                if (tt.leaf(t)) { near[t].push_back(pr[1]); continue; }
                for (int32_t a = 0; a < tt.nchild[t]; ++a) stack.push_back(tt.first_child[t] + a);
            }
        }
    }
    struct Unit { int32_t leaf; int64_t work; std::vector<int32_t> b, e; };
    for (int32_t c = 0; c < tt.ncell(); ++c)
        if (tt.leaf(c)) hp.p2p_leaf.push_back(c);
    // each leaf's units, independent per leaf: slices of the leaves on several threads,
    // concatenated in leaf order
    const size_t nleaf = hp.p2p_leaf.size();
    const int nth = hp.p2p.size() >= ((size_t)1 << 18) ? plan_threads() : 1;
    std::vector<std::vector<Unit>> units_of(nth);
    std::vector<int64_t> inter_of(nth, 0);
    parallel_slices((size_t)nth, nth, [&](size_t j0, size_t j1) {
        for (size_t j = j0; j < j1; ++j) {   // slice j of the leaves
            const size_t l0 = nleaf * j / nth, l1 = nleaf * (j + 1) / nth;
            std::vector<Unit>& units = units_of[j];
            int64_t inter = 0;
            for (size_t lix = l0; lix < l1; ++lix) {
                const int32_t li = (int32_t)lix, c = hp.p2p_leaf[lix];
                auto& v = near[c];
                std::sort(v.begin(), v.end(), [&](int32_t a, int32_t b) { return ts.begin[a] < ts.begin[b]; });
                const int64_t nt = tt.end[c] - tt.begin[c];
                // merged ranges of the leaf, then cut into units of bounded size
                std::vector<int32_t> rb, re;
                for (size_t i = 0; i < v.size(); ++i) {
                    const int32_t b = (int32_t)ts.begin[v[i]], e = (int32_t)ts.end[v[i]];
                    inter += nt * (int64_t)(e - b);
                    if (!re.empty() && re.back() == b) re.back() = e;
                    else { rb.push_back(b); re.push_back(e); }
                }
                Unit u{li, 0, {}, {}};
                int32_t have = 0;
                auto flush = [&]() {
                    if (!u.b.empty()) { u.work = nt * (int64_t)have; units.push_back(u); }
                    u = Unit{li, 0, {}, {}};
                    have = 0;
                };
                for (size_t k = 0; k < rb.size(); ++k) {
                    int32_t b = rb[k];
                    while (b < re[k]) {
                        if (have == kP2PUnitSources || (int)u.b.size() == kP2PUnitRanges) flush();
                        const int32_t take = std::min(re[k] - b, kP2PUnitSources - have);
                        u.b.push_back(b);
                        u.e.push_back(b + take);
                        have += take;
                        b += take;
                    }
                }
                if (u.b.empty() && units_for_leaf_empty(units, li)) {
                    // a leaf without near sources still owns one (empty) unit: its sums are zero
                    units.push_back(Unit{li, 0, {}, {}});
                } else {
                    flush();
                }
            }
            inter_of[j] = inter;
        }
    });
    std::vector<Unit> units;
    for (int j = 0; j < nth; ++j) {
        hp.p2p_interactions += inter_of[j];
        for (Unit& u : units_of[j]) units.push_back(std::move(u));
    }
    // heaviest units first, so that the last blocks to start are short ones
    std::stable_sort(units.begin(), units.end(), [](const Unit& a, const Unit& b) { return a.work > b.work; });
    {
        size_t nr = 0;
        for (const Unit& u : units) nr += u.b.size();
        hp.p2p_sbeg.reserve(nr); hp.p2p_send.reserve(nr); hp.p2p_soff.reserve(nr);
        hp.p2p_unit_leaf.reserve(units.size()); hp.p2p_part.reserve(units.size());
        hp.p2p_unit_off.reserve(units.size() + 1);
    }
    hp.p2p_unit_off.push_back(0);
    std::vector<std::vector<int32_t>> leaf_units(hp.p2p_leaf.size());
    int64_t parts = 0;
    for (size_t ui = 0; ui < units.size(); ++ui) {
        const Unit& u = units[ui];
        hp.p2p_unit_leaf.push_back(u.leaf);
        int32_t acc = 0;
        for (size_t k = 0; k < u.b.size(); ++k) {
            hp.p2p_sbeg.push_back(u.b[k]);
            hp.p2p_send.push_back(u.e[k]);
            hp.p2p_soff.push_back(acc);
            acc += u.e[k] - u.b[k];
        }
        hp.p2p_unit_off.push_back((int32_t)hp.p2p_sbeg.size());
        hp.p2p_part.push_back((int32_t)parts);
        const int32_t c = hp.p2p_leaf[u.leaf];
        parts += tt.end[c] - tt.begin[c];
        leaf_units[u.leaf].push_back((int32_t)ui);
    }
    if (parts > (1LL << 31) - 1) throw std::runtime_error("too many near-field partial sums");
    hp.p2p_parts = parts;
    hp.p2p_leaf_off.push_back(0);
    for (size_t li = 0; li < leaf_units.size(); ++li) {
        // units of a leaf in the order of their sources, so the reduction order is fixed
        auto& lu = leaf_units[li];
        std::sort(lu.begin(), lu.end(), [&](int32_t a, int32_t b) {
            const int32_t ra = hp.p2p_unit_off[a], rb2 = hp.p2p_unit_off[b];
            const int32_t na = hp.p2p_unit_off[a + 1] - ra, nb = hp.p2p_unit_off[b + 1] - rb2;
            const int32_t ka = na ? hp.p2p_sbeg[ra] : -1, kb = nb ? hp.p2p_sbeg[rb2] : -1;
            return ka < kb;
        });
        hp.p2p_leaf_units.insert(hp.p2p_leaf_units.end(), lu.begin(), lu.end());
        hp.p2p_leaf_off.push_back((int32_t)hp.p2p_leaf_units.size());
    }
}

}  // namespace defmm

namespace defmm {

namespace {
template <typename V> void append(std::vector<V>& dst, const std::vector<V>& src) {
    dst.insert(dst.end(), src.begin(), src.end());
}
// dst += src with v -> v + off for v >= 0 (negative entries mark "none" and stay)
template <typename V, typename O> void append_off(std::vector<V>& dst, const std::vector<V>& src, O off) {
    dst.reserve(dst.size() + src.size());
    for (V v : src) dst.push_back(v >= 0 ? (V)(v + off) : v);
}
}  // namespace

void union_host_plans(std::vector<HostPlan>& parts, HostPlan& u) {
    if (parts.empty()) throw std::runtime_error("union of no geometries");
    const HostPlan& f = parts[0];
    for (const HostPlan& h : parts) {
        if (h.p != f.p || h.N != f.N) throw std::runtime_error("union: geometries need the same order and DFT length");
        if (!h.same) throw std::runtime_error("union: sources must equal targets");
    }
    u = HostPlan();
    u.same = true;
    u.p = f.p; u.N = f.N; u.NF = f.NF; u.NFpad = f.NFpad; u.P3 = f.P3;
    u.eta = f.eta; u.hf_kw = f.hf_kw; u.self_eps_rel = f.self_eps_rel; u.damping = f.damping;
    u.radial_power = f.radial_power;
    u.kappa = f.kappa; u.eps_self = f.eps_self; u.d_aabb = f.d_aabb; u.side = f.side;
    for (int a = 0; a < 3; ++a) u.corner[a] = f.corner[a];
    u.lv = f.lv;
    u.m1 = f.m1;
    u.tw = f.tw;
    u.ngeo = (int)parts.size();
    u.geo_point_off.push_back(0);
    u.geo_cell_off.push_back(0);
    u.geo_level_off.push_back(0);
    u.chk_max_blocks = 0;
    std::vector<size_t> m2m_levels, l2l_levels;
    size_t nlev_m2m = 0, nlev_l2l = 0;
    for (const HostPlan& h : parts) {
        nlev_m2m = std::max(nlev_m2m, h.m2m_lvl.size());
        nlev_l2l = std::max(nlev_l2l, h.l2l_lvl.size());
    }
    u.m2m_lvl.assign(nlev_m2m, {});
    u.l2l_lvl.assign(nlev_l2l, {});
    u.l2l_par.assign(nlev_l2l, {});
    u.grp_member_off.push_back(0);
    u.grp_chunk_off.push_back(0);
    u.chk_blk_off.push_back(0);
    u.p2p_unit_off.push_back(0);
    u.p2p_leaf_off.push_back(0);
    for (HostPlan& h : parts) {
        const int64_t pb = u.nx;                               // point base
        const int32_t cb = u.tt.ncell();                       // cell base
        const int32_t lb = u.geo_level_off.back();             // global level base
        const int32_t mb = (int32_t)u.m_cell.size();           // multipole base
        const int32_t eb = (int32_t)u.l_cell.size();           // local expansion base
        const int32_t sb = (int32_t)u.slot_level.size();       // phase-slot base
        const int32_t spb = (int32_t)u.spec_level.size();      // spectrum base
        const int32_t hb = (int32_t)u.m2f_list.size();         // Fourier-multipole base
        const int32_t gb = (int32_t)u.grp_member_off.size() - 1;
        const int32_t gmb = (int32_t)u.grp_members.size();
        const int32_t chb = (int32_t)u.chk_nspec.size();
        const int32_t bb = (int32_t)u.chk_blk.size();
        const int32_t ob = (int32_t)u.chk_op.size();
        const int32_t ub = (int32_t)u.p2p_unit_leaf.size();
        const int32_t rb = (int32_t)u.p2p_sbeg.size();
        const int32_t leb = (int32_t)u.p2p_leaf.size();
        const int32_t lub = (int32_t)u.p2p_leaf_units.size();
        const int64_t partb = u.p2p_parts;
        const int nlev = (int)h.tt.level_range.size();
        // tree (sources = targets)
        Tree& t = u.tt;
        append_off(t.perm, h.tt.perm, pb);
        for (int32_t lv : h.tt.level) t.level.push_back(lv + lb);
        append(t.ix, h.tt.ix); append(t.iy, h.tt.iy); append(t.iz, h.tt.iz);
        append_off(t.begin, h.tt.begin, pb); append_off(t.end, h.tt.end, pb);
        append_off(t.parent, h.tt.parent, cb); append_off(t.first_child, h.tt.first_child, cb);
        append(t.nchild, h.tt.nchild);
        for (int32_t c = 0; c < h.tt.ncell(); ++c) {
            const double s = h.lv.side(h.tt.level[c]);
            u.cell_corner_u.push_back(h.corner[0] + s * h.tt.ix[c]);
            u.cell_corner_u.push_back(h.corner[1] + s * h.tt.iy[c]);
            u.cell_corner_u.push_back(h.corner[2] + s * h.tt.iz[c]);
            u.cell_geo.push_back((int32_t)u.geo_kappa.size());
        }
        for (int l = 0; l < std::max(nlev, 1); ++l) u.level_side_u.push_back(h.lv.side(l));
        for (auto& r : h.m2l) u.m2l.push_back({r[0] + cb, r[1] + cb, r[2]});
        for (auto& r : h.p2p) u.p2p.push_back({r[0] + cb, r[1] + cb});
        // expansions
        append_off(u.m_cell, h.m_cell, cb); append(u.m_dir, h.m_dir);
        append_off(u.m_first, h.m_first, mb); append(u.m_count, h.m_count);
        append_off(u.l_cell, h.l_cell, cb); append(u.l_dir, h.l_dir);
        append_off(u.l_first, h.l_first, eb); append(u.l_count, h.l_count);
        append_off(u.m_slot, h.m_slot, sb); append_off(u.l_slot, h.l_slot, sb);
        for (int32_t lv : h.slot_level) u.slot_level.push_back(lv + lb);
        append(u.slot_dir, h.slot_dir); append(u.slot_u, h.slot_u);
        append(u.slot_P, h.slot_P); append(u.slot_Q, h.slot_Q);
        // spectra
        for (int32_t lv : h.spec_level) u.spec_level.push_back(lv + lb);
        append(u.spec_kbar, h.spec_kbar);
        for (size_t i = 0; i < h.spec_level.size(); ++i) u.spec_kappa.push_back(h.kappa);
        append_off(u.m2f_list, h.m2f_list, mb);
        append_off(u.mhat_of_m, h.mhat_of_m, hb);
        // M2L schedule
        for (size_t i = 1; i < h.grp_member_off.size(); ++i) u.grp_member_off.push_back(h.grp_member_off[i] + gmb);
        append_off(u.grp_members, h.grp_members, eb);
        for (size_t i = 1; i < h.grp_chunk_off.size(); ++i) u.grp_chunk_off.push_back(h.grp_chunk_off[i] + chb);
        for (int32_t code : h.grp_half) u.grp_half.push_back(((code >> 1) + gb) * 2 + (code & 1));
        for (size_t i = 1; i < h.chk_blk_off.size(); ++i) u.chk_blk_off.push_back(h.chk_blk_off[i] + bb);
        append(u.chk_nspec, h.chk_nspec);
        for (size_t cc = 0; cc < h.chk_nspec.size(); ++cc) {   // spectra first, then Fourier multipoles
            const int32_t b0 = h.chk_blk_off[cc], b1 = h.chk_blk_off[cc + 1];
            for (int32_t b = b0; b < b1; ++b)
                u.chk_blk.push_back(h.chk_blk[b] + (b - b0 < h.chk_nspec[cc] ? spb : hb));
        }
        append_off(u.chk_op_off, h.chk_op_off, ob);
        append(u.chk_op, h.chk_op);
        u.chk_max_blocks = std::max(u.chk_max_blocks, h.chk_max_blocks);
        for (int v = 0; v < 3; ++v) u.chk_stage_blocks[v] = std::max(u.chk_stage_blocks[v], h.chk_stage_blocks[v]);
        // upward / downward lists, by local level
        for (size_t l = 0; l < h.m2m_lvl.size(); ++l) append_off(u.m2m_lvl[l], h.m2m_lvl[l], mb);
        for (size_t l = 0; l < h.l2l_lvl.size(); ++l) {
            const int32_t parb = (int32_t)u.l2l_par[l].size();
            const auto& e = h.l2l_lvl[l];
            for (size_t i = 0; i + 3 < e.size(); i += 4) {
                u.l2l_lvl[l].push_back(e[i] + eb);
                u.l2l_lvl[l].push_back(e[i + 1]);
                u.l2l_lvl[l].push_back(e[i + 2] + parb);
                u.l2l_lvl[l].push_back(e[i + 3]);
            }
            append_off(u.l2l_par[l], h.l2l_par[l], eb);
        }
        append_off(u.p2m_cells, h.p2m_cells, cb);
        append_off(u.l2p_cells, h.l2p_cells, cb);
        // near field
        append_off(u.p2p_unit_leaf, h.p2p_unit_leaf, leb);
        for (size_t i = 1; i < h.p2p_unit_off.size(); ++i) u.p2p_unit_off.push_back(h.p2p_unit_off[i] + rb);
        append_off(u.p2p_sbeg, h.p2p_sbeg, (int32_t)pb);
        append_off(u.p2p_send, h.p2p_send, (int32_t)pb);
        append(u.p2p_soff, h.p2p_soff);
        append_off(u.p2p_part, h.p2p_part, (int32_t)partb);
        append_off(u.p2p_leaf, h.p2p_leaf, cb);
        for (size_t i = 1; i < h.p2p_leaf_off.size(); ++i) u.p2p_leaf_off.push_back(h.p2p_leaf_off[i] + lub);
        append_off(u.p2p_leaf_units, h.p2p_leaf_units, ub);
        u.p2p_parts += h.p2p_parts;
        u.p2p_interactions += h.p2p_interactions;
        // per geometry
        u.geo_kappa.push_back(h.kappa);
        u.geo_eps.push_back(h.eps_self);
        for (int a = 0; a < 3; ++a) u.geo_center.push_back(h.corner[a] + h.side / 2);
        u.nx += h.nx;
        u.ny += h.ny;
        u.geo_point_off.push_back(u.nx);
        u.geo_cell_off.push_back(u.tt.ncell());
        u.geo_level_off.push_back(lb + std::max(nlev, 1));
        u.tt.level_range.resize(std::max(u.tt.level_range.size(), (size_t)nlev));
        u.d_aabb = std::max(u.d_aabb, h.d_aabb);
        h = HostPlan();   // release the part
    }
}

}  // namespace defmm
