// Host-side plan construction of the directional equispaced FMM.
//
// Geometry and traversal follow the paper: Ncrit octree on Morton-sorted
// points (Sec. 4.2.1), cube-face direction tree (Sec. 4.1.2), strict and
// directional MACs (Sec. 3.2 footnote, Eq. macdirref), the dual tree
// traversal (Alg. 1), blank DTT (Alg. 2) and blank downward pass (Alg. 3).
// The result is flattened into index tables consumed by the CUDA kernels.
#pragma once

#include <array>
#include <cstdint>
#include <functional>
#include <string>
#include <vector>

namespace defmm {

constexpr int kMaxLevel = 21;
constexpr int kNumLevels = kMaxLevel + 1;
constexpr int kMaxOrder = 8;
constexpr int kP2PUnitSources = 4096;
constexpr int kP2PUnitRanges = 256;

struct Tree {
    std::vector<int64_t> perm;  // sorted position -> input index
    std::vector<int32_t> level, ix, iy, iz;
    std::vector<int64_t> begin, end;
    std::vector<int32_t> parent, first_child, nchild;
    std::vector<std::pair<int32_t, int32_t>> level_range;
    int32_t ncell() const { return (int32_t)level.size(); }
    bool leaf(int32_t c) const { return nchild[c] == 0; }
};

struct Levels {
    double side0 = 1, kappa = 0, eta = 1, hf_kw = 1;
    bool hf[kNumLevels + 1] = {};
    int l_hf = -1;
    double side(int l) const;
    double radius(int l) const;
    bool mac(int l, int64_t kx, int64_t ky, int64_t kz) const;
    void mac_terms(int l, double* A2, double* F) const;   // directional MAC: A2 <= F * S
    int E(int l) const { return l_hf - l; }
};

// Directions (Sec. 4.1.2): face f in +x,-x,+y,-y,+z,-z, sub-square (i, j).
int64_t num_directions(int E);
void direction_vector(int E, int64_t d, double out[3]);
int64_t direction_father(int E, int64_t d);
int64_t direction_negate(int E, int64_t d);
int64_t best_direction(int E, int64_t kx, int64_t ky, int64_t kz);

// Canonical offset and the signed permutation taking it to k (Sec. 4.3).
// kbar = |k| sorted decreasingly (ties: lower axis first); sigma[i] is the
// position of axis i; sign[i] = sign(k_i) (+1 for 0).  code = perm_id*8 + mask.
struct Canon {
    int kbar[3];
    int sigma[3];
    int sign[3];
};
Canon canonical(int64_t kx, int64_t ky, int64_t kz);
int transform_code(const Canon& c);

struct HostPlan {
    // parameters
    int64_t nx = 0, ny = 0;
    bool same = true;
    double kappa = 0;
    double damping = 0;   // lambda of the kernel exp((i kappa - lambda) r) / (4 pi r^P)
    int radial_power = 1; // P, 1 or 2
    int p = 4, N = 7, NF = 343, NFpad = 344, P3 = 64;
    double eta = 1, hf_kw = 1, self_eps_rel = 1e-10;
    double eps_self = 0, d_aabb = 0, side = 0;
    double corner[3] = {0, 0, 0};
    Levels lv;
    Tree tt, ts_own;
    const Tree& ts() const { return same ? tt : ts_own; }

    // traversal output
    std::vector<std::array<int32_t, 3>> m2l;  // t, s, direction (-1: LF)
    std::vector<std::array<int32_t, 2>> p2p;  // t, s
    std::vector<std::vector<int32_t>> marks_t, marks_s;

    // effective expansions (cell, dir), level-major, Morton within a level
    std::vector<int32_t> m_cell, m_dir, m_first, m_count;  // multipole, source tree
    std::vector<int32_t> l_cell, l_dir, l_first, l_count;  // local, target tree
    std::vector<int32_t> m_slot, l_slot;                   // phase-table slot, -1 for LF

    // phase slots: one per (level, direction) used
    std::vector<int32_t> slot_level, slot_dir;
    std::vector<double> slot_u;  // 3 per slot
    std::vector<double> slot_P;  // [slot][axis][a] complex (2 doubles)
    std::vector<double> slot_Q;  // [slot][axis][octbit][b] complex

    // 1-D son->father interpolation matrices M1[o][a][b] (Sec. 5.2.1)
    std::vector<double> m1;
    // twiddles e^{2 pi i m / N}
    std::vector<double> tw;

    // spectra: (level, kbar)
    std::vector<int32_t> spec_level;
    std::vector<std::array<int32_t, 3>> spec_kbar;

    // M2F: multipole ids that are M2L sources, and inverse map
    std::vector<int32_t> m2f_list, mhat_of_m;

    // M2L work schedule.  A group is the set of sibling target expansions that
    // share a father cell and a direction (at most 8 members).  Its pairs are
    // cut into chunks; a chunk names the distinct blocks it needs (canonical
    // spectra, then Fourier multipoles: one TMA stage) and its pair operations,
    // sorted by member.  Groups are ordered by work, heaviest first.
    std::vector<int32_t> grp_member_off, grp_members;   // CSR: group -> local expansion ids
    std::vector<int32_t> grp_chunk_off;                 // CSR: group -> chunks
    std::vector<int32_t> grp_half;                      // blocks of <= 4 members: group * 2 + half
    std::vector<int32_t> chk_blk_off, chk_nspec;        // CSR: chunk -> blocks; spectra first
    std::vector<int32_t> chk_blk;                       // spectrum id or Fourier-multipole slot
    std::vector<int32_t> chk_op_off;                    // 9 per chunk: op ranges of members 0..7, end
    std::vector<int32_t> chk_op;                        // spec_blk | mhat_blk << 8 | code << 16
    int32_t chk_max_blocks = 0;
    // largest stage in blocks when RB = 1, 2, 4 right-hand sides share it:
    // max over chunks of (spectra + RB * multipoles)
    int32_t chk_stage_blocks[3] = {0, 0, 0};

    // M2M per level (parent level l): entries of 9 ints: parent exp, 8 child exps (-1)
    std::vector<std::vector<int32_t>> m2m_lvl;
    // L2L per level (child level l): entries child exp, octant, par_first, par_count
    std::vector<std::vector<int32_t>> l2l_lvl;
    std::vector<std::vector<int32_t>> l2l_par;  // parent local exp ids per level
    // leaves
    std::vector<int32_t> p2m_cells, l2p_cells;  // cells (source / target tree)
    // P2P work units: a unit is one target leaf against at most kP2PUnitSources
    // of its near sources (its ranges in Morton order); units are ordered by
    // work, heaviest first.  Each unit writes partial sums for its leaf's
    // targets at p2p_part[unit]; the leaf's units are reduced in order.
    std::vector<int32_t> p2p_unit_leaf;              // unit -> index into p2p_leaf
    std::vector<int32_t> p2p_unit_off;               // CSR into the unit ranges below
    std::vector<int32_t> p2p_sbeg, p2p_send, p2p_soff;  // ranges, prefix within the unit
    std::vector<int32_t> p2p_part;                   // unit -> first partial-sum slot
    std::vector<int32_t> p2p_leaf;                   // target leaf cells
    std::vector<int32_t> p2p_leaf_off, p2p_leaf_units;  // leaf -> its units, in source order
    int64_t p2p_parts = 0;                           // partial-sum slots per right-hand side
    int64_t p2p_interactions = 0;

    int64_t nM() const { return (int64_t)m_cell.size(); }
    int64_t nL() const { return (int64_t)l_cell.size(); }

    // Union of several geometries (ngeo > 1, see union_host_plans): every table
    // above is the concatenation of the geometries' own, indices offset; cell
    // levels are global level ids (geometry g's level l is geo_level_off[g] + l)
    // and the per-geometry quantities live here.  Empty for one geometry.
    int ngeo = 1;
    std::vector<int64_t> geo_point_off;     // ngeo + 1, points (sorted and caller order)
    std::vector<int32_t> geo_cell_off;      // ngeo + 1, cells
    std::vector<int32_t> geo_level_off;     // ngeo + 1, global level ids
    std::vector<double> geo_kappa, geo_eps, geo_center;   // per geometry (center: 3 each)
    std::vector<double> level_side_u;       // per global level
    std::vector<double> cell_corner_u;      // 3 per cell
    std::vector<int32_t> cell_geo;          // per cell
    std::vector<double> spec_kappa;         // per spectrum
};

// Concatenates independently built plans (same order, DFT length, options;
// sources = targets) into one: the application phase of the union runs every
// phase as one launch over all geometries.  parts are consumed.
void union_host_plans(std::vector<HostPlan>& parts, HostPlan& out);

// Plan files (persist.cpp): the host plan and the coordinates it was built
// from (caller order; Y empty when sources = targets).  Throw on failure.
void save_plan_file(const std::string& path, const HostPlan& hp, const std::vector<double>& X,
                    const std::vector<double>& Y);
void load_plan_file(const std::string& path, HostPlan& hp, std::vector<double>& X, std::vector<double>& Y);

// A replacement for the trees, the dual tree traversal and the marks of
// Alg. 2: given hp with its cube and levels set, fills hp.tt (hp.ts_own),
// hp.m2l, hp.p2p, hp.marks_t and hp.marks_s as the host construction would
// (the marks may already be deduplicated).
using FrontEnd = std::function<void(HostPlan&)>;

// Builds everything above from host coordinates (Y == nullptr: same tree).
// The traversal is breadth first: pairs of a level in order, son pairs in
// (a, b) order.  With `front`, the trees, traversal and marks come from it.
// Throws std::runtime_error with a message on invalid input.
void build_host_plan(const double* X, int64_t nx, const double* Y, int64_t ny, double kappa,
                     int order, int leaf, double eta, double hf_kw, int fft_n, double self_eps,
                     int chunk_blocks, HostPlan& hp, const FrontEnd* front = nullptr);

}  // namespace defmm
