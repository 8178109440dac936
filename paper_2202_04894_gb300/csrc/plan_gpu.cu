// Device construction of the plan's front end: bounding-cube Morton keys and
// their stable sort, the Ncrit octree level by level (Sec. 4.2.1), the dual
// tree traversal (Alg. 1) breadth first, the best direction of every
// high-frequency M2L offset (Sec. 4.2.3), and the blank DTT + blank downward
// pass (Alg. 2, Alg. 3).  The tables it returns are those of the host
// construction in plan.cpp, entry for entry (the same integer rules, the
// same floating-point expressions for quantisation and the MAC), so the rest
// of the plan is built from either.
//
// Building blocks, all written here: an exclusive prefix sum over int64
// counts (block scans, recursive over block sums) and a stable least
// significant digit radix sort of 64-bit keys with 64-bit values (8-bit
// digits; within a tile the rank of an item among equal digits is counted in
// input order with warp match masks).  Lists whose order matters are
// produced by count -> exclusive scan -> write, never by atomics, so every
// table is deterministic.
#include <cuda_runtime.h>

#include <algorithm>
#include <cstdlib>
#include <cstdint>
#include <stdexcept>
#include <string>
#include <vector>

#include "plan.h"
#include "plan_gpu.h"

namespace defmm {
namespace {

// ------------------------------------------------------------ device buffers
template <typename V> struct DBuf {
    V* p = nullptr;
    int64_t n = 0;
    DBuf() = default;
    DBuf(const DBuf&) = delete;
    DBuf& operator=(const DBuf&) = delete;
    DBuf(DBuf&& o) noexcept { swap(o); }
    DBuf& operator=(DBuf&& o) noexcept { swap(o); return *this; }
    ~DBuf() { if (p) cudaFree(p); }
    void alloc(int64_t count) {
        if (p) cudaFree(p);
        p = nullptr;
        n = count;
        if (count > 0 && cudaMalloc(&p, sizeof(V) * (size_t)count) != cudaSuccess) {
            cudaGetLastError();
            throw DeviceFailure("device allocation failed while building the plan", true);
        }
    }
    void swap(DBuf& o) { std::swap(p, o.p); std::swap(n, o.n); }
};

void ck(cudaError_t e, const char* what) {
    if (e != cudaSuccess)
        throw DeviceFailure(std::string("plan construction on the device: ") + what + ": " + cudaGetErrorString(e),
                            e == cudaErrorMemoryAllocation);
}

unsigned grid_for(int64_t n, int threads) {
    const int64_t g = (n + threads - 1) / threads;
    return (unsigned)std::max<int64_t>(1, std::min<int64_t>(g, 1 << 30));
}

// ------------------------------------------------------------ exclusive scan
constexpr int kScanThreads = 256, kScanItems = 4, kScanTile = kScanThreads * kScanItems;

// out[i] = sum of in[0..i) within each tile of kScanTile; sums[tile] = the tile's total
__global__ void k_scan_tiles(const int64_t* __restrict__ in, int64_t* __restrict__ out, int64_t* __restrict__ sums,
                             int64_t n) {
    __shared__ int64_t warp_tot[kScanThreads / 32];
    const int64_t base = (int64_t)blockIdx.x * kScanTile + (int64_t)threadIdx.x * kScanItems;
    int64_t v[kScanItems], t = 0;
#pragma unroll
    for (int j = 0; j < kScanItems; ++j) {
        v[j] = base + j < n ? in[base + j] : 0;
        t += v[j];
    }
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    int64_t incl = t;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const int64_t y = __shfl_up_sync(0xffffffffu, incl, o);
        if (lane >= o) incl += y;
    }
    if (lane == 31) warp_tot[warp] = incl;
    __syncthreads();
    int64_t before = 0;
    for (int w = 0; w < warp; ++w) before += warp_tot[w];
    int64_t run = before + incl - t;
#pragma unroll
    for (int j = 0; j < kScanItems; ++j) {
        if (base + j < n) out[base + j] = run;
        run += v[j];
    }
    if (threadIdx.x == kScanThreads - 1) sums[blockIdx.x] = before + incl;
}

__global__ void k_scan_add(int64_t* __restrict__ out, const int64_t* __restrict__ add, int64_t n) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) out[i] += add[i / kScanTile];
}

// out = exclusive prefix sum of in (n entries; in and out may alias); returns the total
int64_t scan_excl(const int64_t* in, int64_t* out, int64_t n, cudaStream_t st) {
    if (n <= 0) return 0;
    const int64_t tiles = (n + kScanTile - 1) / kScanTile;
    DBuf<int64_t> sums, sums_x;
    sums.alloc(tiles);
    sums_x.alloc(tiles);
    k_scan_tiles<<<(unsigned)tiles, kScanThreads, 0, st>>>(in, out, sums.p, n);
    ck(cudaGetLastError(), "scan");
    int64_t total = 0;
    if (tiles > 1) {
        total = scan_excl(sums.p, sums_x.p, tiles, st);
        k_scan_add<<<grid_for(n, 256), 256, 0, st>>>(out, sums_x.p, n);
        ck(cudaGetLastError(), "scan add");
    } else {
        ck(cudaMemcpyAsync(&total, sums.p, sizeof(int64_t), cudaMemcpyDeviceToHost, st), "scan total");
        ck(cudaStreamSynchronize(st), "scan total");
    }
    return total;
}

// ------------------------------------------------------------ stable radix sort
constexpr int kSortThreads = 256, kSortItems = 8, kSortTile = kSortThreads * kSortItems;

__global__ void k_radix_hist(const uint64_t* __restrict__ key, int64_t n, int shift, int64_t tiles,
                             int64_t* __restrict__ hist) {
    __shared__ int cnt[256];
    cnt[threadIdx.x] = 0;
    __syncthreads();
    const int64_t base = (int64_t)blockIdx.x * kSortTile;
    for (int j = threadIdx.x; j < kSortTile; j += kSortThreads)
        if (base + j < n) atomicAdd(&cnt[(key[base + j] >> shift) & 255], 1);
    __syncthreads();
    hist[(int64_t)threadIdx.x * tiles + blockIdx.x] = cnt[threadIdx.x];   // digit-major
}

// Scatters a tile's items to their places: offs[d * tiles + tile] is where the
// tile's first item of digit d goes; items of equal digit keep their order.
__global__ void k_radix_scatter(const uint64_t* __restrict__ key, const int64_t* __restrict__ val, int64_t n,
                                int shift, int64_t tiles, const int64_t* __restrict__ offs,
                                uint64_t* __restrict__ key_out, int64_t* __restrict__ val_out) {
    __shared__ int64_t run[256];
    __shared__ int wcnt[kSortThreads / 32][256];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    run[threadIdx.x] = offs[(int64_t)threadIdx.x * tiles + blockIdx.x];
    const int64_t base = (int64_t)blockIdx.x * kSortTile;
    for (int ch = 0; ch < kSortItems; ++ch) {
        for (int w = 0; w < kSortThreads / 32; ++w) wcnt[w][threadIdx.x] = 0;
        __syncthreads();
        const int64_t i = base + (int64_t)ch * kSortThreads + threadIdx.x;
        const bool have = i < n;
        const int d = have ? (int)((key[i] >> shift) & 255) : 256 + lane;   // absent items: unique dummies
        const unsigned peers = __match_any_sync(0xffffffffu, d);
        const int rank = __popc(peers & ((1u << lane) - 1));
        if (have && rank == 0) wcnt[warp][d] = __popc(peers);
        __syncthreads();
        if (have) {
            int64_t pos = run[d] + rank;
            for (int w = 0; w < warp; ++w) pos += wcnt[w][d];
            key_out[pos] = key[i];
            val_out[pos] = val[i];
        }
        __syncthreads();
        int add = 0;
        for (int w = 0; w < kSortThreads / 32; ++w) add += wcnt[w][threadIdx.x];
        run[threadIdx.x] += add;
        __syncthreads();
    }
}

// Sorts (key, val) by key, stably, over the low `bits` bits of the keys.
void radix_sort(DBuf<uint64_t>& key, DBuf<int64_t>& val, int64_t n, int bits, cudaStream_t st) {
    if (n <= 1) return;
    const int64_t tiles = (n + kSortTile - 1) / kSortTile;
    DBuf<uint64_t> k2;
    DBuf<int64_t> v2, hist;
    k2.alloc(n);
    v2.alloc(n);
    hist.alloc(256 * tiles);
    for (int shift = 0; shift < bits; shift += 8) {
        k_radix_hist<<<(unsigned)tiles, kSortThreads, 0, st>>>(key.p, n, shift, tiles, hist.p);
        ck(cudaGetLastError(), "radix histogram");
        scan_excl(hist.p, hist.p, 256 * tiles, st);
        k_radix_scatter<<<(unsigned)tiles, kSortThreads, 0, st>>>(key.p, val.p, n, shift, tiles, hist.p, k2.p, v2.p);
        ck(cudaGetLastError(), "radix scatter");
        key.swap(k2);
        val.swap(v2);
    }
}


// ------------------------------------------------------------ Morton keys and the octree
// Quantisation to 21 bits per axis inside the cube and bit interleaving
// (x lowest), with the host construction's expression.
__global__ void k_morton(const double* __restrict__ P, int64_t n, double c0, double c1, double c2, double side,
                         uint64_t* __restrict__ key, int64_t* __restrict__ idx) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const double scale = (double)(1LL << kMaxLevel);
    const int64_t gmax = (1LL << kMaxLevel) - 1;
    const double corner[3] = {c0, c1, c2};
    int64_t g[3];
    for (int a = 0; a < 3; ++a) {
        const double v = __dmul_rn(__ddiv_rn(__dsub_rn(P[3 * i + a], corner[a]), side), scale);
        const int64_t q = (int64_t)floor(v);
        g[a] = q < 0 ? 0 : (q > gmax ? gmax : q);
    }
    uint64_t k = 0;
    for (int b = 0; b < kMaxLevel; ++b)
        for (int a = 0; a < 3; ++a) k |= (uint64_t)((g[a] >> b) & 1) << (3 * b + a);
    key[i] = k;
    idx[i] = i;
}

// Children of the cells [0, ncell) of one level: a cell with more than ncrit
// points (below the deepest level) is split into its non-empty octants, in
// octant order.  bnd: 9 boundaries per cell; cnt: non-empty octants.
__global__ void k_split_count(const uint64_t* __restrict__ skey, const int64_t* __restrict__ beg,
                              const int64_t* __restrict__ end, int64_t ncell, int lev, int ncrit,
                              int64_t* __restrict__ bnd, int64_t* __restrict__ cnt) {
    const int64_t c = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (c >= ncell) return;
    const int64_t b = beg[c], e = end[c];
    int64_t nch = 0;
    int64_t* bd = bnd + 9 * c;
    if (e - b > ncrit && lev < kMaxLevel) {
        const int shift = 3 * (kMaxLevel - lev - 1);
        const uint64_t base = (skey[b] >> shift) >> 3 << 3;
        int64_t lo = b;
        bd[0] = b;
        for (int o = 0; o < 8; ++o) {
            // first index in [lo, e) whose prefix exceeds base + o
            int64_t L = lo, H = e;
            while (L < H) {
                const int64_t mid = L + (H - L) / 2;
                if ((skey[mid] >> shift) > base + (uint64_t)o) H = mid; else L = mid + 1;
            }
            bd[o + 1] = L;
            if (L > lo) ++nch;
            lo = L;
        }
    }
    cnt[c] = nch;
}

struct LevelCells {   // one level's cells on the device
    DBuf<int64_t> beg, end;
    DBuf<int32_t> ix, iy, iz, parent;
};

__global__ void k_split_write(const int64_t* __restrict__ bnd, const int64_t* __restrict__ cnt,
                              const int64_t* __restrict__ off, int64_t ncell, int32_t first_id,
                              int32_t next_first_id, const int32_t* __restrict__ ix, const int32_t* __restrict__ iy,
                              const int32_t* __restrict__ iz, int32_t* __restrict__ first_child,
                              int32_t* __restrict__ nchild, int64_t* __restrict__ cb, int64_t* __restrict__ ce,
                              int32_t* __restrict__ cx, int32_t* __restrict__ cy, int32_t* __restrict__ cz,
                              int32_t* __restrict__ cpar) {
    const int64_t c = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (c >= ncell) return;
    const int64_t n = cnt[c];
    first_child[c] = n > 0 ? next_first_id + (int32_t)off[c] : -1;
    nchild[c] = (int32_t)n;
    if (n == 0) return;
    const int64_t* bd = bnd + 9 * c;
    int64_t j = off[c];
    for (int o = 0; o < 8; ++o) {
        if (bd[o + 1] == bd[o]) continue;
        cb[j] = bd[o];
        ce[j] = bd[o + 1];
        cx[j] = 2 * ix[c] + (o & 1);
        cy[j] = 2 * iy[c] + ((o >> 1) & 1);
        cz[j] = 2 * iz[c] + ((o >> 2) & 1);
        cpar[j] = first_id + (int32_t)c;
        ++j;
    }
}

template <typename V> void to_host(std::vector<V>& dst, const V* src, int64_t n, cudaStream_t st) {
    const size_t at = dst.size();
    dst.resize(at + (size_t)n);
    if (n > 0) ck(cudaMemcpyAsync(dst.data() + at, src, sizeof(V) * (size_t)n, cudaMemcpyDeviceToHost, st), "copy back");
}

// The octree of n points (host array P), as plan.cpp's build_tree makes it.
void device_tree(const double* P, int64_t n, const double corner[3], double side, int ncrit, Tree& t,
                 cudaStream_t st) {
    DBuf<double> dP;
    dP.alloc(3 * n);
    ck(cudaMemcpyAsync(dP.p, P, sizeof(double) * 3 * (size_t)n, cudaMemcpyHostToDevice, st), "points");
    DBuf<uint64_t> key;
    DBuf<int64_t> idx;
    key.alloc(n);
    idx.alloc(n);
    k_morton<<<grid_for(n, 256), 256, 0, st>>>(dP.p, n, corner[0], corner[1], corner[2], side, key.p, idx.p);
    ck(cudaGetLastError(), "morton keys");
    radix_sort(key, idx, n, 3 * kMaxLevel, st);
    t.perm.clear();
    to_host(t.perm, idx.p, n, st);

    t.level = {0}; t.ix = {0}; t.iy = {0}; t.iz = {0};
    t.begin = {0}; t.end = {n}; t.parent = {-1};
    t.first_child.clear(); t.nchild.clear(); t.level_range.clear();
    LevelCells cur;
    cur.beg.alloc(1); cur.end.alloc(1); cur.ix.alloc(1); cur.iy.alloc(1); cur.iz.alloc(1);
    const int64_t zero = 0;
    const int32_t zi = 0;
    ck(cudaMemcpyAsync(cur.beg.p, &zero, sizeof(int64_t), cudaMemcpyHostToDevice, st), "root");
    ck(cudaMemcpyAsync(cur.end.p, &n, sizeof(int64_t), cudaMemcpyHostToDevice, st), "root");
    for (auto* a : {cur.ix.p, cur.iy.p, cur.iz.p})
        ck(cudaMemcpyAsync(a, &zi, sizeof(int32_t), cudaMemcpyHostToDevice, st), "root");
    int64_t ncur = 1;
    int32_t first = 0;
    for (int lev = 0; ncur > 0; ++lev) {
        t.level_range.push_back({first, first + (int32_t)ncur});
        DBuf<int64_t> bnd, cnt, off;
        bnd.alloc(9 * ncur);
        cnt.alloc(ncur);
        off.alloc(ncur);
        k_split_count<<<grid_for(ncur, 128), 128, 0, st>>>(key.p, cur.beg.p, cur.end.p, ncur, lev, ncrit, bnd.p, cnt.p);
        ck(cudaGetLastError(), "split count");
        const int64_t nnext = scan_excl(cnt.p, off.p, ncur, st);
        if ((int64_t)first + ncur + nnext > (int64_t(1) << 31) - 2) throw std::runtime_error("too many octree cells");
        LevelCells nxt;
        nxt.beg.alloc(nnext); nxt.end.alloc(nnext); nxt.ix.alloc(nnext); nxt.iy.alloc(nnext); nxt.iz.alloc(nnext);
        nxt.parent.alloc(nnext);
        DBuf<int32_t> fc, nc;
        fc.alloc(ncur);
        nc.alloc(ncur);
        const int32_t next_first = first + (int32_t)ncur;
        k_split_write<<<grid_for(ncur, 128), 128, 0, st>>>(bnd.p, cnt.p, off.p, ncur, first, next_first, cur.ix.p,
                                                           cur.iy.p, cur.iz.p, fc.p, nc.p, nxt.beg.p, nxt.end.p,
                                                           nxt.ix.p, nxt.iy.p, nxt.iz.p, nxt.parent.p);
        ck(cudaGetLastError(), "split write");
        to_host(t.first_child, fc.p, ncur, st);
        to_host(t.nchild, nc.p, ncur, st);
        to_host(t.begin, nxt.beg.p, nnext, st);
        to_host(t.end, nxt.end.p, nnext, st);
        to_host(t.ix, nxt.ix.p, nnext, st);
        to_host(t.iy, nxt.iy.p, nnext, st);
        to_host(t.iz, nxt.iz.p, nnext, st);
        to_host(t.parent, nxt.parent.p, nnext, st);
        ck(cudaStreamSynchronize(st), "tree level");
        t.level.resize(t.level.size() + (size_t)nnext, lev + 1);
        cur.beg.swap(nxt.beg); cur.end.swap(nxt.end);
        cur.ix.swap(nxt.ix); cur.iy.swap(nxt.iy); cur.iz.swap(nxt.iz);
        first = next_first;
        ncur = nnext;
    }
}

// ------------------------------------------------------------ dual tree traversal (Alg. 1), breadth first
struct DevTree {   // what the traversal and the blank passes read of a tree
    DBuf<int32_t> ix, iy, iz, first_child, nchild;
    void upload(const Tree& t, cudaStream_t st) {
        const int64_t n = t.ncell();
        ix.alloc(n); iy.alloc(n); iz.alloc(n); first_child.alloc(n); nchild.alloc(n);
        ck(cudaMemcpyAsync(ix.p, t.ix.data(), 4 * (size_t)n, cudaMemcpyHostToDevice, st), "tree");
        ck(cudaMemcpyAsync(iy.p, t.iy.data(), 4 * (size_t)n, cudaMemcpyHostToDevice, st), "tree");
        ck(cudaMemcpyAsync(iz.p, t.iz.data(), 4 * (size_t)n, cudaMemcpyHostToDevice, st), "tree");
        ck(cudaMemcpyAsync(first_child.p, t.first_child.data(), 4 * (size_t)n, cudaMemcpyHostToDevice, st), "tree");
        ck(cudaMemcpyAsync(nchild.p, t.nchild.data(), 4 * (size_t)n, cudaMemcpyHostToDevice, st), "tree");
    }
};

// The MAC of one level with the host's expressions: high frequency,
// A^2 <= F * S with A = max(kappa w^2, 2w), F = eta^2 s^2 and S the integer
// squared gap; low frequency, max |k_i| >= 2.
struct MacLevel {
    int hf;
    double A2, F;
};

__device__ __forceinline__ bool mac_dev(const MacLevel& m, int64_t kx, int64_t ky, int64_t kz) {
    const int64_t ax = kx < 0 ? -kx : kx, ay = ky < 0 ? -ky : ky, az = kz < 0 ? -kz : kz;
    if (m.hf) {
        const int64_t gx = ax > 1 ? ax - 1 : 0, gy = ay > 1 ? ay - 1 : 0, gz = az > 1 ? az - 1 : 0;
        const int64_t S = gx * gx + gy * gy + gz * gz;
        return m.A2 <= __dmul_rn(m.F, (double)S);
    }
    return max(ax, max(ay, az)) >= 2;
}

// Pair kinds of one frontier: 0 M2L (MAC holds), 1 P2P (a leaf), 2 recurse.
__global__ void k_dtt_classify(const int32_t* __restrict__ ft, const int32_t* __restrict__ fs, int64_t nf,
                               MacLevel mac, const int32_t* __restrict__ tix, const int32_t* __restrict__ tiy,
                               const int32_t* __restrict__ tiz, const int32_t* __restrict__ tnc,
                               const int32_t* __restrict__ six, const int32_t* __restrict__ siy,
                               const int32_t* __restrict__ siz, const int32_t* __restrict__ snc,
                               int64_t* __restrict__ n_m2l, int64_t* __restrict__ n_p2p, int64_t* __restrict__ n_kid) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= nf) return;
    const int32_t t = ft[i], s = fs[i];
    const int64_t kx = (int64_t)tix[t] - six[s], ky = (int64_t)tiy[t] - siy[s], kz = (int64_t)tiz[t] - siz[s];
    int64_t a = 0, b = 0, k = 0;
    if (mac_dev(mac, kx, ky, kz)) a = 1;
    else if (tnc[t] == 0 || snc[s] == 0) b = 1;
    else k = (int64_t)tnc[t] * snc[s];
    n_m2l[i] = a;
    n_p2p[i] = b;
    n_kid[i] = k;
}

__global__ void k_dtt_write(const int32_t* __restrict__ ft, const int32_t* __restrict__ fs, int64_t nf,
                            const int64_t* __restrict__ o_m2l, const int64_t* __restrict__ o_p2p,
                            const int64_t* __restrict__ o_kid, const int64_t* __restrict__ n_m2l,
                            const int64_t* __restrict__ n_p2p, const int64_t* __restrict__ n_kid,
                            const int32_t* __restrict__ tfc, const int32_t* __restrict__ sfc,
                            const int32_t* __restrict__ snc, int32_t* __restrict__ m2l, int32_t* __restrict__ p2p,
                            int32_t* __restrict__ kt, int32_t* __restrict__ ks) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= nf) return;
    const int32_t t = ft[i], s = fs[i];
    if (n_m2l[i]) {
        m2l[2 * o_m2l[i]] = t;
        m2l[2 * o_m2l[i] + 1] = s;
    } else if (n_p2p[i]) {
        p2p[2 * o_p2p[i]] = t;
        p2p[2 * o_p2p[i] + 1] = s;
    } else if (n_kid[i]) {   // son pairs in (a, b) order
        const int32_t ns = snc[s];
        int64_t j = o_kid[i];
        const int64_t na = n_kid[i] / ns;
        for (int64_t a = 0; a < na; ++a)
            for (int32_t b = 0; b < ns; ++b, ++j) {
                kt[j] = tfc[t] + (int32_t)a;
                ks[j] = sfc[s] + b;
            }
    }
}

// Breadth-first Alg. 1 from (root, root): the pairs of level l are handled in
// frontier order, each producing an M2L pair, a P2P pair or its son pairs (the
// next frontier).  The M2L pairs of every level stay on the device (levels in
// order, pairs of a level in frontier order) for the direction and mark passes;
// the P2P pairs go to hp.p2p.
struct LevelPairs {
    int level;
    int64_t n;
    DBuf<int32_t> pr;   // 2 per pair: target cell, source cell
};

void device_dtt(const DevTree& dt, const DevTree& ds, const std::vector<MacLevel>& macs, HostPlan& hp,
                std::vector<LevelPairs>& m2l_levels, cudaStream_t st) {
    DBuf<int32_t> ft, fs;
    ft.alloc(1);
    fs.alloc(1);
    const int32_t zero = 0;
    ck(cudaMemcpyAsync(ft.p, &zero, 4, cudaMemcpyHostToDevice, st), "frontier");
    ck(cudaMemcpyAsync(fs.p, &zero, 4, cudaMemcpyHostToDevice, st), "frontier");
    int64_t nf = 1, total = 0;
    std::vector<int32_t> pbuf;
    for (int l = 0; nf > 0; ++l) {
        if (l >= (int)macs.size()) throw std::runtime_error("internal: traversal deeper than the trees");
        DBuf<int64_t> nm, np, nk, om, op, ok;
        nm.alloc(nf); np.alloc(nf); nk.alloc(nf); om.alloc(nf); op.alloc(nf); ok.alloc(nf);
        k_dtt_classify<<<grid_for(nf, 256), 256, 0, st>>>(ft.p, fs.p, nf, macs[l], dt.ix.p, dt.iy.p, dt.iz.p,
                                                          dt.nchild.p, ds.ix.p, ds.iy.p, ds.iz.p, ds.nchild.p, nm.p,
                                                          np.p, nk.p);
        ck(cudaGetLastError(), "traversal classify");
        const int64_t cm = scan_excl(nm.p, om.p, nf, st);
        const int64_t cp = scan_excl(np.p, op.p, nf, st);
        const int64_t ck_ = scan_excl(nk.p, ok.p, nf, st);
        total += cm;
        if (total > (int64_t(1) << 31) - 2) throw std::runtime_error("too many M2L pairs");
        m2l_levels.emplace_back();
        LevelPairs& lp = m2l_levels.back();
        lp.level = l;
        lp.n = cm;
        lp.pr.alloc(2 * cm);
        DBuf<int32_t> p2p, kt, ks;
        p2p.alloc(2 * cp); kt.alloc(ck_); ks.alloc(ck_);
        k_dtt_write<<<grid_for(nf, 256), 256, 0, st>>>(ft.p, fs.p, nf, om.p, op.p, ok.p, nm.p, np.p, nk.p,
                                                       dt.first_child.p, ds.first_child.p, ds.nchild.p, lp.pr.p, p2p.p,
                                                       kt.p, ks.p);
        ck(cudaGetLastError(), "traversal write");
        pbuf.clear();
        to_host(pbuf, p2p.p, 2 * cp, st);
        ck(cudaStreamSynchronize(st), "traversal level");
        for (int64_t j = 0; j < cp; ++j) hp.p2p.push_back({pbuf[2 * j], pbuf[2 * j + 1]});
        ft.swap(kt);
        fs.swap(ks);
        nf = ck_;
    }
}

// ------------------------------------------------------------ best directions (Sec. 4.2.3)
// Integer direction vectors of the cube-face direction tree with E
// subdivisions (face f = +x,-x,+y,-y,+z,-z; sub-square (i, j)), as plan.cpp.
__device__ void direction_int_dev(int E, int64_t d, int64_t w[3]) {
    const int64_t n = 1LL << E;
    const int64_t f = d / (n * n), rem = d % (n * n);
    const int64_t i = rem / n, j = rem % n;
    const int m = (int)(f / 2);
    const int64_t sign = (f % 2 == 0) ? 1 : -1;
    const int m1 = (m == 0) ? 1 : 0, m2 = (m == 2) ? 1 : 2;
    w[m] = sign * n;
    w[m1] = 2 * i + 1 - n;
    w[m2] = 2 * j + 1 - n;
}

__device__ int64_t direction_negate_dev(int E, int64_t d) {
    const int64_t n = 1LL << E;
    const int64_t f = d / (n * n), rem = d % (n * n);
    const int64_t i = rem / n, j = rem % n;
    return (f ^ 1) * n * n + (n - 1 - i) * n + (n - 1 - j);
}

// (dot, n2, d) candidates: larger dot^2 / n2 first (exactly, in 128-bit
// integers), then the lower index; dot <= 0 never wins.
struct Cand {
    int64_t d, dot, n2;
};
__device__ __forceinline__ bool better(const Cand& a, const Cand& b) {   // a before b
    if (a.d < 0) return false;
    if (b.d < 0) return true;
    const __int128 lhs = (__int128)a.dot * a.dot * b.n2, rhs = (__int128)b.dot * b.dot * a.n2;
    if (lhs != rhs) return lhs > rhs;
    return a.d < b.d;
}

// One block per distinct (level, offset): argmax over the level's directions
// of <v, k>/|v| for k whose first non-zero entry is positive, the negation of
// the choice for -k otherwise (so u(-k) = -u(k)).
__global__ void k_best_direction(const uint64_t* __restrict__ okey, int64_t nk, int B, int64_t K0,
                                 const int* __restrict__ level_E, int32_t* __restrict__ out) {
    __shared__ Cand red[256];
    const int64_t q = blockIdx.x;
    if (q >= nk) return;
    const uint64_t key = okey[q];
    const uint64_t mask = (1ULL << B) - 1;
    const int l = (int)(key >> (3 * B));
    int64_t kx = (int64_t)((key >> (2 * B)) & mask) - K0, ky = (int64_t)((key >> B) & mask) - K0,
            kz = (int64_t)(key & mask) - K0;
    const int E = level_E[l];
    const int64_t first = kx != 0 ? kx : (ky != 0 ? ky : kz);
    const bool neg = first <= 0;
    if (neg) { kx = -kx; ky = -ky; kz = -kz; }
    const int64_t nd = 6LL << (2 * E);
    Cand best{-1, 0, 1};
    for (int64_t d = threadIdx.x; d < nd; d += blockDim.x) {
        int64_t w[3];
        direction_int_dev(E, d, w);
        const int64_t dot = w[0] * kx + w[1] * ky + w[2] * kz;
        if (dot <= 0) continue;
        const Cand c{d, dot, w[0] * w[0] + w[1] * w[1] + w[2] * w[2]};
        if (better(c, best)) best = c;
    }
    red[threadIdx.x] = best;
    __syncthreads();
    for (int h = blockDim.x / 2; h > 0; h >>= 1) {
        if (threadIdx.x < h && better(red[threadIdx.x + h], red[threadIdx.x])) red[threadIdx.x] = red[threadIdx.x + h];
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        const int64_t d = red[0].d;
        out[q] = (int32_t)(neg && d >= 0 ? direction_negate_dev(E, d) : d);
    }
}

// Offset keys of the high-frequency M2L pairs: (level, kx + K0, ky + K0, kz + K0), B bits each
__global__ void k_offset_keys(const int32_t* __restrict__ pr, const int32_t* __restrict__ plev, int64_t n,
                              const int32_t* __restrict__ tix, const int32_t* __restrict__ tiy,
                              const int32_t* __restrict__ tiz, const int32_t* __restrict__ six,
                              const int32_t* __restrict__ siy, const int32_t* __restrict__ siz, int B, int64_t K0,
                              uint64_t* __restrict__ key, int64_t* __restrict__ idx) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const int32_t t = pr[2 * i], s = pr[2 * i + 1];
    const uint64_t kx = (uint64_t)((int64_t)tix[t] - six[s] + K0), ky = (uint64_t)((int64_t)tiy[t] - siy[s] + K0),
                   kz = (uint64_t)((int64_t)tiz[t] - siz[s] + K0);
    key[i] = ((uint64_t)plev[i] << (3 * B)) | (kx << (2 * B)) | (ky << B) | kz;
    idx[i] = i;
}

__global__ void k_fill_level(int32_t* __restrict__ lev, int64_t n, int32_t l) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) lev[i] = l;
}

// max over the pairs of max(|tx - sx|, |ty - sy|, |tz - sz|), into *out (zeroed by the caller)
__global__ void k_max_offset(const int32_t* __restrict__ pr, int64_t n, const int32_t* __restrict__ tix,
                             const int32_t* __restrict__ tiy, const int32_t* __restrict__ tiz,
                             const int32_t* __restrict__ six, const int32_t* __restrict__ siy,
                             const int32_t* __restrict__ siz, unsigned long long* __restrict__ out) {
    unsigned long long m = 0;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        const int32_t t = pr[2 * i], s = pr[2 * i + 1];
        const int64_t ax = llabs((int64_t)tix[t] - six[s]), ay = llabs((int64_t)tiy[t] - siy[s]),
                      az = llabs((int64_t)tiz[t] - siz[s]);
        m = max(m, (unsigned long long)max(ax, max(ay, az)));
    }
    for (int o = 16; o > 0; o >>= 1) m = max(m, __shfl_xor_sync(0xffffffffu, m, o));
    if ((threadIdx.x & 31) == 0) atomicMax(out, m);
}

// first[i] = 1 where sorted key i differs from key i - 1
__global__ void k_first_of_run(const uint64_t* __restrict__ key, int64_t n, int64_t* __restrict__ first) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) first[i] = (i == 0 || key[i] != key[i - 1]) ? 1 : 0;
}

__global__ void k_compact_runs(const uint64_t* __restrict__ key, const int64_t* __restrict__ first,
                               const int64_t* __restrict__ pos, int64_t n, uint64_t* __restrict__ ukey) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n && first[i]) ukey[pos[i]] = key[i];
}

// direction of sorted pair i: its run's direction, written at the pair's own position
__global__ void k_scatter_dir(const int64_t* __restrict__ idx, const int64_t* __restrict__ first,
                              const int64_t* __restrict__ pos, int64_t n, const int32_t* __restrict__ udir,
                              int32_t* __restrict__ dir) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) dir[idx[i]] = udir[pos[i] + first[i] - 1];
}

// Sorted distinct keys of key[0..n) (the runs of the sorted array), on the device
int64_t sorted_unique(DBuf<uint64_t>& key, DBuf<int64_t>& idx, int64_t n, int bits, DBuf<int64_t>& first,
                      DBuf<int64_t>& pos, DBuf<uint64_t>& ukey, cudaStream_t st) {
    radix_sort(key, idx, n, bits, st);
    first.alloc(n);
    pos.alloc(n);
    k_first_of_run<<<grid_for(n, 256), 256, 0, st>>>(key.p, n, first.p);
    ck(cudaGetLastError(), "runs");
    const int64_t nu = scan_excl(first.p, pos.p, n, st);
    ukey.alloc(nu);
    k_compact_runs<<<grid_for(n, 256), 256, 0, st>>>(key.p, first.p, pos.p, n, ukey.p);
    ck(cudaGetLastError(), "compact");
    return nu;
}

// (cell << 27 | direction) of one end of every high-frequency M2L pair
__global__ void k_mark_keys(const int32_t* __restrict__ pr, const int32_t* __restrict__ dir, int64_t n, int side,
                            uint64_t* __restrict__ key, int64_t* __restrict__ idx) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    key[i] = ((uint64_t)pr[2 * i + side] << 27) | (uint64_t)dir[i];
    idx[i] = i;
}

}  // namespace

// ------------------------------------------------------------ the front end
void device_front(const double* X, int64_t nx, const double* Y, int64_t ny, int ncrit, HostPlan& hp,
                  cudaStream_t st, double* device_ms) {
    struct Events {   // released on every exit
        cudaEvent_t a = nullptr, b = nullptr;
        ~Events() {
            if (a) cudaEventDestroy(a);
            if (b) cudaEventDestroy(b);
        }
    } ev;
    ck(cudaEventCreate(&ev.a), "event");
    ck(cudaEventCreate(&ev.b), "event");
    ck(cudaEventRecord(ev.a, st), "event");
    device_tree(X, nx, hp.corner, hp.side, ncrit, hp.tt, st);
    if (Y) device_tree(Y, ny, hp.corner, hp.side, ncrit, hp.ts_own, st);
    const Tree& tt = hp.tt;
    const Tree& ts = hp.ts();
    DevTree dt, ds_own;
    dt.upload(tt, st);
    if (Y) ds_own.upload(ts, st);
    const DevTree& ds = Y ? ds_own : dt;

    std::vector<MacLevel> macs(kNumLevels + 1);
    for (int l = 0; l <= kNumLevels; ++l) {
        macs[l].hf = hp.lv.hf[l] ? 1 : 0;
        hp.lv.mac_terms(l, &macs[l].A2, &macs[l].F);
    }
    hp.m2l.clear();
    hp.p2p.clear();
    std::vector<LevelPairs> levels;
    device_dtt(dt, ds, macs, hp, levels, st);

    // the high-frequency pairs, concatenated on the device in level order
    int64_t nh = 0, nall = 0;
    for (const LevelPairs& lp : levels) {
        nall += lp.n;
        if (hp.lv.hf[lp.level]) nh += lp.n;
    }
    hp.marks_t.assign(tt.ncell(), {});
    hp.marks_s.assign(ts.ncell(), {});
    std::vector<int32_t> dir;
    if (nh > 0) {
        DBuf<int32_t> dpr, dlev, ddir;
        dpr.alloc(2 * nh);
        dlev.alloc(nh);
        ddir.alloc(nh);
        int64_t o = 0;
        for (const LevelPairs& lp : levels) {
            if (!hp.lv.hf[lp.level] || lp.n == 0) continue;
            ck(cudaMemcpyAsync(dpr.p + 2 * o, lp.pr.p, 8 * (size_t)lp.n, cudaMemcpyDeviceToDevice, st), "pairs");
            k_fill_level<<<grid_for(lp.n, 256), 256, 0, st>>>(dlev.p + o, lp.n, lp.level);
            ck(cudaGetLastError(), "pair levels");
            o += lp.n;
        }
        DBuf<unsigned long long> dk;
        dk.alloc(1);
        ck(cudaMemsetAsync(dk.p, 0, sizeof(unsigned long long), st), "offsets");
        k_max_offset<<<std::min<unsigned>(grid_for(nh, 256), 4096), 256, 0, st>>>(
            dpr.p, nh, dt.ix.p, dt.iy.p, dt.iz.p, ds.ix.p, ds.iy.p, ds.iz.p, dk.p);
        ck(cudaGetLastError(), "offsets");
        std::vector<unsigned long long> kv;
        to_host(kv, dk.p, 1, st);
        ck(cudaStreamSynchronize(st), "offsets");
        const int64_t kmax = (int64_t)kv[0];
        int B = 1;
        while ((int64_t(1) << B) < 2 * kmax + 1) ++B;
        if (5 + 3 * B > 64) throw std::runtime_error("M2L offsets too large for the device plan");
        // directions: one search per distinct (level, offset)
        DBuf<uint64_t> key, ukey;
        DBuf<int64_t> idx, first, pos;
        key.alloc(nh);
        idx.alloc(nh);
        k_offset_keys<<<grid_for(nh, 256), 256, 0, st>>>(dpr.p, dlev.p, nh, dt.ix.p, dt.iy.p, dt.iz.p, ds.ix.p,
                                                         ds.iy.p, ds.iz.p, B, kmax, key.p, idx.p);
        ck(cudaGetLastError(), "offset keys");
        const int64_t nu = sorted_unique(key, idx, nh, (5 + 3 * B + 7) / 8 * 8, first, pos, ukey, st);
        std::vector<int> levE(kNumLevels + 1, 0);
        for (int l = 0; l <= kNumLevels; ++l) levE[l] = hp.lv.hf[l] ? hp.lv.E(l) : 0;
        DBuf<int> dE;
        dE.alloc(kNumLevels + 1);
        ck(cudaMemcpyAsync(dE.p, levE.data(), sizeof(int) * levE.size(), cudaMemcpyHostToDevice, st), "levels");
        DBuf<int32_t> udir;
        udir.alloc(nu);
        k_best_direction<<<(unsigned)nu, 256, 0, st>>>(ukey.p, nu, B, kmax, dE.p, udir.p);
        ck(cudaGetLastError(), "best directions");
        k_scatter_dir<<<grid_for(nh, 256), 256, 0, st>>>(idx.p, first.p, pos.p, nh, udir.p, ddir.p);
        ck(cudaGetLastError(), "directions");
        to_host(dir, ddir.p, nh, st);
        // Alg. 2 marks, deduplicated on the device: (cell, direction) of each end of the pairs
        std::vector<uint64_t> marks[2];
        for (int side = 0; side < 2; ++side) {
            DBuf<uint64_t> mk, umk;
            DBuf<int64_t> mi, mf, mp;
            mk.alloc(nh);
            mi.alloc(nh);
            k_mark_keys<<<grid_for(nh, 256), 256, 0, st>>>(dpr.p, ddir.p, nh, side, mk.p, mi.p);
            ck(cudaGetLastError(), "mark keys");
            const int64_t nm = sorted_unique(mk, mi, nh, 64, mf, mp, umk, st);
            to_host(marks[side], umk.p, nm, st);
            ck(cudaStreamSynchronize(st), "marks");
        }
        for (uint64_t k : marks[0]) hp.marks_t[(size_t)(k >> 27)].push_back((int32_t)(k & ((1u << 27) - 1)));
        for (uint64_t k : marks[1]) hp.marks_s[(size_t)(k >> 27)].push_back((int32_t)(k & ((1u << 27) - 1)));
    }
    // the M2L list in traversal order: direction -1 on low-frequency levels
    hp.m2l.resize((size_t)nall);
    std::vector<int32_t> pbuf;
    int64_t at = 0, oh = 0;
    for (const LevelPairs& lp : levels) {
        if (lp.n == 0) continue;
        pbuf.clear();
        to_host(pbuf, lp.pr.p, 2 * lp.n, st);
        ck(cudaStreamSynchronize(st), "pairs");
        const bool hf = hp.lv.hf[lp.level];
        for (int64_t j = 0; j < lp.n; ++j) {
            const int32_t d = hf ? dir[(size_t)(oh + j)] : -1;
            if (hf && d < 0) throw std::runtime_error("internal: no direction for an M2L offset");
            hp.m2l[(size_t)(at + j)] = {pbuf[2 * j], pbuf[2 * j + 1], d};
        }
        at += lp.n;
        if (hf) oh += lp.n;
    }
    ck(cudaEventRecord(ev.b, st), "event");
    ck(cudaEventSynchronize(ev.b), "event");
    float ms = 0.f;
    ck(cudaEventElapsedTime(&ms, ev.a, ev.b), "event");
    if (device_ms) *device_ms = ms;
}

}  // namespace defmm
