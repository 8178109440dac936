// C ABI of the library (include/defmm.h): plan creation (one geometry or a
// union of several), upload, workspaces, applies, tuning and shards.
#include <cuda_runtime.h>

#include <algorithm>
#include <chrono>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <mutex>
#include <new>
#include <stdexcept>
#include <string>
#include <vector>

#include "defmm.h"
#include "kernels.cuh"
#include "plan.h"
#include "plan_gpu.h"
#include "plan_state.h"

namespace defmm {
template <typename T> cudaError_t configure_kernels();
}

using namespace defmm;

namespace {

thread_local std::string g_err;

defmm_status fail(defmm_status s, const std::string& msg) {
    g_err = msg;
    return s;
}

defmm_status cuda_fail(cudaError_t e, const char* what) {
    if (e == cudaErrorMemoryAllocation) {
        cudaGetLastError();
        return fail(DEFMM_ERR_OOM, std::string(what) + ": " + cudaGetErrorString(e));
    }
    return fail(DEFMM_ERR_CUDA, std::string(what) + ": " + cudaGetErrorString(e));
}

}  // namespace

defmm_status defmm::set_error(defmm_status s, const std::string& msg) { return fail(s, msg); }

namespace {

#define CK(call, what)                                     \
    do {                                                   \
        cudaError_t e_ = (call);                           \
        if (e_ != cudaSuccess) return cuda_fail(e_, what); \
    } while (0)

// Host image of the plan tables, 256-byte aligned, copied to the device once.
struct Blob {
    std::vector<unsigned char> bytes;
    template <typename V> size_t add(const V* src, size_t count) {
        size_t off = (bytes.size() + 255) / 256 * 256;
        bytes.resize(off + count * sizeof(V));
        if (count) std::memcpy(bytes.data() + off, src, count * sizeof(V));
        return off;
    }
    template <typename V> size_t add(const std::vector<V>& v) { return add(v.data(), v.size()); }
};

}  // namespace

namespace {

bool is_device_ptr(const void* p) {
    cudaPointerAttributes a;
    if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    return a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged;
}

defmm_status read_points(const double* P, int64_t n, std::vector<double>& out, bool host_only) {
    out.resize(3 * (size_t)n);
    if (!host_only && is_device_ptr(P)) {
        CK(cudaMemcpy(out.data(), P, out.size() * sizeof(double), cudaMemcpyDeviceToHost), "copy points to host");
    } else {
        std::memcpy(out.data(), P, out.size() * sizeof(double));
    }
    return DEFMM_OK;
}

template <typename T> size_t workspace_bytes(const HostPlan& hp, int R) {
    size_t c = sizeof(typename Cplx<T>::type);
    return c * R * ((size_t)hp.ny + hp.nx + (size_t)hp.nM() * hp.P3 + hp.m2f_list.size() * (size_t)hp.NFpad +
                    (size_t)hp.nL() * hp.P3 + (size_t)hp.p2p_parts);
}

template <typename T> defmm_status ensure_workspace(defmm_plan_s* pl, Workspace<T>& w, int R, bool host) {
    const HostPlan& hp = pl->hp;
    if (w.R < R) {
        size_t need = workspace_bytes<T>(hp, R);
        if (pl->hbm_budget && pl->arena_bytes + need > pl->hbm_budget)
            return fail(DEFMM_ERR_OOM, "workspace exceeds hbm_budget");
        w.release();
        using C = typename Cplx<T>::type;
        CK(cudaMalloc(&w.qs, sizeof(C) * R * (size_t)hp.ny), "workspace qs");
        CK(cudaMalloc(&w.ps, sizeof(C) * R * (size_t)hp.nx), "workspace ps");
        CK(cudaMalloc(&w.M, sizeof(C) * R * (size_t)std::max<int64_t>(1, hp.nM()) * hp.P3), "workspace M");
        CK(cudaMalloc(&w.Mhat, sizeof(C) * R * std::max<size_t>(1, hp.m2f_list.size()) * hp.NFpad), "workspace Mhat");
        CK(cudaMalloc(&w.L, sizeof(C) * R * (size_t)std::max<int64_t>(1, hp.nL()) * hp.P3), "workspace L");
        CK(cudaMalloc(&w.part, sizeof(C) * R * (size_t)std::max<int64_t>(1, hp.p2p_parts)), "workspace near-field partials");
        w.R = R;
        w.bytes = need;
    }
    if (host && !w.q_stage) {
        using C = typename Cplx<T>::type;
        CK(cudaMalloc(&w.q_stage, sizeof(C) * w.R * (size_t)hp.ny), "staging q");
        CK(cudaMalloc(&w.p_stage, sizeof(C) * w.R * (size_t)hp.nx), "staging p");
    }
    return DEFMM_OK;
}

// Builds the device image of the plan and forms the spectra on the GPU.
defmm_status upload(defmm_plan_s* pl, const std::vector<double>& X, const std::vector<double>& Y,
                    cudaStream_t stream) {
    HostPlan& hp = pl->hp;
    const Tree& tt = hp.tt;
    const Tree& ts = hp.ts();
    Blob b;

    // sorted coordinates and permutations
    std::vector<double> Xs(3 * (size_t)hp.nx);
    for (int64_t i = 0; i < hp.nx; ++i)
        for (int a = 0; a < 3; ++a) Xs[3 * i + a] = X[3 * tt.perm[i] + a];
    size_t o_Xs = b.add(Xs), o_Ys = o_Xs;
    if (!hp.same) {
        std::vector<double> Ys(3 * (size_t)hp.ny);
        for (int64_t i = 0; i < hp.ny; ++i)
            for (int a = 0; a < 3; ++a) Ys[3 * i + a] = Y[3 * ts.perm[i] + a];
        o_Ys = b.add(Ys);
    }
    size_t o_pt = b.add(tt.perm), o_ps = hp.same ? o_pt : b.add(ts.perm);
    // single-precision coordinates as hi + lo pairs relative to the cube centre
    auto split4 = [&](const std::vector<double>& src, int64_t n, const Tree& tr, size_t& oh, size_t& ol) {
        std::vector<float4> hi(n), lo(n);
        double c0[3] = {hp.corner[0] + hp.side / 2, hp.corner[1] + hp.side / 2, hp.corner[2] + hp.side / 2};
        int g = 0;   // geometry of sorted point i (a union: relative to that geometry's cube centre)
        for (int64_t i = 0; i < n; ++i) {
            if (hp.ngeo > 1) {
                while (i >= hp.geo_point_off[g + 1]) ++g;
                for (int a = 0; a < 3; ++a) c0[a] = hp.geo_center[3 * g + a];
            }
            float h[3], l[3];
            for (int a = 0; a < 3; ++a) {
                double d = src[3 * tr.perm[i] + a] - c0[a];
                h[a] = (float)d;
                l[a] = (float)(d - (double)h[a]);
            }
            hi[i] = make_float4(h[0], h[1], h[2], 0.f);
            lo[i] = make_float4(l[0], l[1], l[2], 0.f);
        }
        oh = b.add(hi);
        ol = b.add(lo);
    };
    size_t o_Xh, o_Xl, o_Yh, o_Yl;
    split4(X, hp.nx, tt, o_Xh, o_Xl);
    if (hp.same) { o_Yh = o_Xh; o_Yl = o_Xl; }
    else split4(Y, hp.ny, ts, o_Yh, o_Yl);

    auto cells = [&](const Tree& tr, size_t& ob, size_t& oe, size_t& ol, size_t& oc) {
        std::vector<int32_t> beg(tr.ncell()), end(tr.ncell());
        std::vector<double> cor(3 * (size_t)tr.ncell());
        for (int32_t c = 0; c < tr.ncell(); ++c) {
            beg[c] = (int32_t)tr.begin[c];
            end[c] = (int32_t)tr.end[c];
            if (hp.ngeo > 1) {   // a union: each geometry's own cube
                for (int a = 0; a < 3; ++a) cor[3 * c + a] = hp.cell_corner_u[3 * c + a];
                continue;
            }
            double s = hp.lv.side(tr.level[c]);
            cor[3 * c] = hp.corner[0] + s * tr.ix[c];
            cor[3 * c + 1] = hp.corner[1] + s * tr.iy[c];
            cor[3 * c + 2] = hp.corner[2] + s * tr.iz[c];
        }
        ob = b.add(beg); oe = b.add(end); ol = b.add(tr.level); oc = b.add(cor);
    };
    size_t o_ctb, o_cte, o_ctl, o_ctc, o_csb, o_cse, o_csl, o_csc;
    cells(tt, o_ctb, o_cte, o_ctl, o_ctc);
    if (hp.same) { o_csb = o_ctb; o_cse = o_cte; o_csl = o_ctl; o_csc = o_ctc; }
    else cells(ts, o_csb, o_cse, o_csl, o_csc);
    std::vector<double> lside(kNumLevels);
    for (int l = 0; l < kNumLevels; ++l) lside[l] = hp.lv.side(l);
    if (hp.ngeo > 1) lside = hp.level_side_u;   // global level ids of a union
    size_t o_lside = b.add(lside);
    size_t o_cgeo = 0, o_gk = 0, o_ge = 0, o_spk = 0;
    if (hp.ngeo > 1) {
        o_cgeo = b.add(hp.cell_geo); o_gk = b.add(hp.geo_kappa); o_ge = b.add(hp.geo_eps);
        o_spk = b.add(hp.spec_kappa);
    }
    const int32_t zero_flag[4] = {0, 0, 0, 0};
    size_t o_err = b.add(zero_flag, 4);

    size_t o_mf = b.add(hp.m_first), o_mc = b.add(hp.m_count), o_ms = b.add(hp.m_slot);
    size_t o_lf = b.add(hp.l_first), o_lc = b.add(hp.l_count), o_ls = b.add(hp.l_slot);
    size_t o_su = b.add(hp.slot_u);
    size_t o_m2f = b.add(hp.m2f_list);
    size_t o_gmo = b.add(hp.grp_member_off), o_gm = b.add(hp.grp_members), o_gco = b.add(hp.grp_chunk_off);
    size_t o_ghf = b.add(hp.grp_half);
    std::vector<int32_t> gbig, gsmall, gmid, glarge;   // the splits by group size
    for (size_t g = 0; g + 1 < hp.grp_member_off.size(); ++g) {
        const int nm = hp.grp_member_off[g + 1] - hp.grp_member_off[g];
        if (nm > 4) gbig.push_back((int32_t)g);
        else gsmall.push_back((int32_t)(2 * g));
        if (nm > 7) glarge.push_back((int32_t)g);
        else if (nm > 4) gmid.push_back((int32_t)g);
    }
    size_t o_gbig = b.add(gbig), o_gsmall = b.add(gsmall), o_gmid = b.add(gmid), o_glarge = b.add(glarge);
    size_t o_cbo = b.add(hp.chk_blk_off), o_cns = b.add(hp.chk_nspec), o_cb = b.add(hp.chk_blk);
    size_t o_coo = b.add(hp.chk_op_off), o_co = b.add(hp.chk_op);
    size_t o_p2m = b.add(hp.p2m_cells), o_l2p = b.add(hp.l2p_cells);
    size_t o_pul = b.add(hp.p2p_unit_leaf), o_puo = b.add(hp.p2p_unit_off), o_psb = b.add(hp.p2p_sbeg),
           o_pse = b.add(hp.p2p_send), o_pso = b.add(hp.p2p_soff), o_ppt = b.add(hp.p2p_part);
    size_t o_pl = b.add(hp.p2p_leaf), o_plo = b.add(hp.p2p_leaf_off), o_plu = b.add(hp.p2p_leaf_units);
    std::vector<size_t> o_m2m(hp.m2m_lvl.size()), o_l2l(hp.l2l_lvl.size()), o_l2lp(hp.l2l_par.size());
    for (size_t l = 0; l < hp.m2m_lvl.size(); ++l) o_m2m[l] = b.add(hp.m2m_lvl[l]);
    for (size_t l = 0; l < hp.l2l_lvl.size(); ++l) { o_l2l[l] = b.add(hp.l2l_lvl[l]); o_l2lp[l] = b.add(hp.l2l_par[l]); }

    // precision-specific tables
    std::vector<float> slotP_f(hp.slot_P.begin(), hp.slot_P.end()), slotQ_f(hp.slot_Q.begin(), hp.slot_Q.end());
    std::vector<float> m1_f(hp.m1.begin(), hp.m1.end()), tw_f(hp.tw.begin(), hp.tw.end());
    size_t o_Pd = b.add(hp.slot_P), o_Qd = b.add(hp.slot_Q), o_m1d = b.add(hp.m1), o_twd = b.add(hp.tw);
    size_t o_Pf = b.add(slotP_f), o_Qf = b.add(slotQ_f), o_m1f = b.add(m1_f), o_twf = b.add(tw_f);
    std::vector<int32_t> kbar(3 * hp.spec_kbar.size());
    for (size_t i = 0; i < hp.spec_kbar.size(); ++i)
        for (int a = 0; a < 3; ++a) kbar[3 * i + a] = hp.spec_kbar[i][a];
    size_t o_sl = b.add(hp.spec_level), o_sk = b.add(kbar);
    size_t nspec = hp.spec_level.size();
    size_t o_specd = b.add((const double2*)nullptr, 0);
    b.bytes.resize(o_specd + nspec * hp.NFpad * sizeof(double2));
    size_t o_specf = b.add((const float2*)nullptr, 0);
    b.bytes.resize(o_specf + nspec * hp.NFpad * sizeof(float2));

    size_t total = b.bytes.size();
    if (pl->hbm_budget && total + workspace_bytes<float>(hp, 1) > pl->hbm_budget)
        return fail(DEFMM_ERR_OOM, "plan exceeds hbm_budget");
    CK(cudaMalloc(&pl->arena, total), "plan tables");
    pl->arena_bytes = total;
    CK(cudaMemcpyAsync(pl->arena, b.bytes.data(), o_specd, cudaMemcpyHostToDevice, stream), "upload plan tables");
    unsigned char* base = pl->arena;
    auto P = [&](size_t off) { return (void*)(base + off); };

    DevCommon& c = pl->common;
    c.p = hp.p; c.N = hp.N; c.NF = hp.NF; c.NFpad = hp.NFpad; c.P3 = hp.P3;
    c.nx = hp.nx; c.ny = hp.ny; c.kappa = hp.kappa; c.eps_self = hp.eps_self; c.damping = hp.damping;
    c.radial_power = hp.radial_power;
    if (hp.ngeo > 1) {
        c.cell_geo = (const int32_t*)P(o_cgeo);
        c.geo_kappa = (const double*)P(o_gk);
        c.geo_eps = (const double*)P(o_ge);
    }
    c.Xs = (const double*)P(o_Xs); c.Ys = (const double*)P(o_Ys);
    c.perm_t = (const int64_t*)P(o_pt); c.perm_s = (const int64_t*)P(o_ps);
    c.Xh = (const float4*)P(o_Xh); c.Xl = (const float4*)P(o_Xl);
    c.Yh = (const float4*)P(o_Yh); c.Yl = (const float4*)P(o_Yl);
    c.ct_beg = (const int32_t*)P(o_ctb); c.ct_end = (const int32_t*)P(o_cte);
    c.ct_level = (const int32_t*)P(o_ctl); c.ct_corner = (const double*)P(o_ctc);
    c.cs_beg = (const int32_t*)P(o_csb); c.cs_end = (const int32_t*)P(o_cse);
    c.cs_level = (const int32_t*)P(o_csl); c.cs_corner = (const double*)P(o_csc);
    c.level_side = (const double*)P(o_lside);
    c.err_flag = (int*)P(o_err);
    c.n_cell_t = hp.tt.ncell(); c.n_cell_s = hp.ts().ncell();
    c.n_mult = hp.nM(); c.n_local = hp.nL();
    c.n_slot = (int64_t)hp.slot_level.size(); c.n_spec = (int64_t)hp.spec_level.size();
    c.n_leaf_all = (int64_t)hp.p2p_leaf.size();
    c.m_first = (const int32_t*)P(o_mf); c.m_count = (const int32_t*)P(o_mc); c.m_slot = (const int32_t*)P(o_ms);
    c.l_first = (const int32_t*)P(o_lf); c.l_count = (const int32_t*)P(o_lc); c.l_slot = (const int32_t*)P(o_ls);
    c.slot_u = (const double*)P(o_su);
    c.m2f_list = (const int32_t*)P(o_m2f); c.n_m2f = (int64_t)hp.m2f_list.size();
    c.grp_member_off = (const int32_t*)P(o_gmo); c.grp_members = (const int32_t*)P(o_gm);
    c.grp_chunk_off = (const int32_t*)P(o_gco);
    c.n_grp = (int64_t)hp.grp_member_off.size() - 1;
    c.grp_half = (const int32_t*)P(o_ghf); c.n_grp_half = (int64_t)hp.grp_half.size();
    c.grp_big = (const int32_t*)P(o_gbig); c.n_grp_big = (int64_t)gbig.size();
    c.grp_small = (const int32_t*)P(o_gsmall); c.n_grp_small = (int64_t)gsmall.size();
    c.grp_mid = (const int32_t*)P(o_gmid); c.n_grp_mid = (int64_t)gmid.size();
    c.grp_large = (const int32_t*)P(o_glarge); c.n_grp_large = (int64_t)glarge.size();
    c.chk_blk_off = (const int32_t*)P(o_cbo); c.chk_nspec = (const int32_t*)P(o_cns); c.chk_blk = (const int32_t*)P(o_cb);
    c.chk_op_off = (const int32_t*)P(o_coo); c.chk_op = (const int32_t*)P(o_co);
    c.chk_max_blocks = hp.chk_max_blocks;
    for (int v = 0; v < 3; ++v) c.chk_stage_blocks[v] = hp.chk_stage_blocks[v];
    for (int v = 0; v < 3; ++v) c.chk_stage_small[v] = 0;
    for (size_t g = 0; g + 1 < hp.grp_member_off.size(); ++g) {
        if (hp.grp_member_off[g + 1] - hp.grp_member_off[g] > 4) continue;
        for (int32_t ch = hp.grp_chunk_off[g]; ch < hp.grp_chunk_off[g + 1]; ++ch) {
            const int32_t nb = hp.chk_blk_off[ch + 1] - hp.chk_blk_off[ch], nsp = hp.chk_nspec[ch];
            for (int v = 0; v < 3; ++v) c.chk_stage_small[v] = std::max(c.chk_stage_small[v], nsp + (1 << v) * (nb - nsp));
        }
    }
    c.m2l_rb = 0;
    c.m2l_members = 0;
    c.p2p_tc_min_rhs = 0;
    // Largest near-field phase in turns, kappa |x - y| / (2 pi), over the P2P cell
    // pairs: |x - y| is at most the largest distance between the two cells' boxes.
    {
        auto corner = [&](const Tree& tr, int32_t cell, int a) {
            if (hp.ngeo > 1) return hp.cell_corner_u[3 * (size_t)cell + a];
            const int32_t i = a == 0 ? tr.ix[cell] : (a == 1 ? tr.iy[cell] : tr.iz[cell]);
            return hp.corner[a] + lside[tr.level[cell]] * i;
        };
        double turns = 0;
        for (const auto& pr : hp.p2p) {
            const double st = lside[tt.level[pr[0]]], ss = lside[ts.level[pr[1]]];
            double d2 = 0;
            for (int a = 0; a < 3; ++a) {
                const double ta = corner(tt, pr[0], a), sa = corner(ts, pr[1], a);
                const double far = std::max(std::fabs(ta + st - sa), std::fabs(sa + ss - ta));
                d2 += far * far;
            }
            const double kap = hp.ngeo > 1 ? hp.geo_kappa[hp.cell_geo[pr[0]]] : hp.kappa;
            turns = std::max(turns, kap * std::sqrt(d2) / (2 * M_PI));
        }
        c.p2p_direct_phase = turns <= 45.0 ? 1 : 0;   // kappa r <= 90 pi
    }
    c.p2m_cells = (const int32_t*)P(o_p2m); c.n_p2m = (int64_t)hp.p2m_cells.size();
    c.l2p_cells = (const int32_t*)P(o_l2p); c.n_l2p = (int64_t)hp.l2p_cells.size();
    c.p2p_unit_leaf = (const int32_t*)P(o_pul); c.p2p_unit_off = (const int32_t*)P(o_puo);
    c.p2p_sbeg = (const int32_t*)P(o_psb); c.p2p_send = (const int32_t*)P(o_pse);
    c.p2p_soff = (const int32_t*)P(o_pso); c.p2p_part = (const int32_t*)P(o_ppt);
    c.n_p2p_units = (int64_t)hp.p2p_unit_leaf.size(); c.p2p_parts = hp.p2p_parts;
    c.p2p_leaf = (const int32_t*)P(o_pl); c.p2p_leaf_off = (const int32_t*)P(o_plo);
    c.p2p_leaf_units = (const int32_t*)P(o_plu);
    c.n_p2p_leaf = (int64_t)hp.p2p_leaf.size();

    pl->m2m.resize(hp.m2m_lvl.size());
    for (size_t l = 0; l < hp.m2m_lvl.size(); ++l)
        pl->m2m[l] = {(const int32_t*)P(o_m2m[l]), (int64_t)hp.m2m_lvl[l].size() / 9};
    pl->l2l.resize(hp.l2l_lvl.size());
    pl->l2l_par.resize(hp.l2l_lvl.size());
    for (size_t l = 0; l < hp.l2l_lvl.size(); ++l) {
        pl->l2l[l] = {(const int32_t*)P(o_l2l[l]), (int64_t)hp.l2l_lvl[l].size() / 4};
        pl->l2l_par[l] = (const int32_t*)P(o_l2lp[l]);
    }
    pl->td.slot_P = (const double2*)P(o_Pd); pl->td.slot_Q = (const double2*)P(o_Qd);
    pl->td.m1 = (const double*)P(o_m1d); pl->td.tw = (const double2*)P(o_twd);
    pl->td.spec = (const double2*)P(o_specd);
    pl->tf.slot_P = (const float2*)P(o_Pf); pl->tf.slot_Q = (const float2*)P(o_Qf);
    pl->tf.m1 = (const float*)P(o_m1f); pl->tf.tw = (const float2*)P(o_twf);
    pl->tf.spec = (const float2*)P(o_specf);

    cudaError_t e = launch_spectra((const int32_t*)P(o_sl), (const int32_t*)P(o_sk), (int)nspec,
                                   (const double*)P(o_lside), hp.p, hp.N, hp.NFpad, hp.kappa,
                                   hp.ngeo > 1 ? (const double*)P(o_spk) : nullptr, hp.damping, hp.radial_power,
                                   (double2*)P(o_specd), (float2*)P(o_specf), stream);
    if (e != cudaSuccess) return cuda_fail(e, "spectra kernel");
    CK(cudaStreamSynchronize(stream), "plan creation");
    return DEFMM_OK;
}

const DevTyped<float>& typed_tables(const defmm_plan_s* pl, float*) { return pl->tf; }
const DevTyped<double>& typed_tables(const defmm_plan_s* pl, double*) { return pl->td; }

std::once_flag g_config_once;
cudaError_t g_config_err = cudaSuccess;

template <typename T> defmm_status apply_impl(defmm_plan_s* pl, Workspace<T>& w, const void* q, void* p,
                                               int nrhs, cudaStream_t stream, void* slice = nullptr,
                                               int64_t slice_ld = 0) {
    defmm_status s = ensure_workspace<T>(pl, w, nrhs, false);
    if (s != DEFMM_OK) return s;
    DevWork<T> dw;
    dw.R = nrhs; dw.qs = w.qs; dw.ps = w.ps; dw.M = w.M; dw.Mhat = w.Mhat; dw.L = w.L; dw.nL = pl->hp.nL();
    dw.part = w.part;
    dw.slice = static_cast<typename Cplx<T>::type*>(slice);
    dw.slice_ld = slice_ld;
    const DevTyped<T>& typed = typed_tables(pl, (T*)nullptr);
    int launches = 0;
    const LevelList* l2l = nullptr;
    const DevCommon c = apply_tables(pl, &l2l);
    cudaError_t e = launch_apply<T>(c, typed, dw, pl->m2m.data(), (int)pl->m2m.size(), l2l,
                                    pl->l2l_par.data(), (int)pl->l2l.size(), q, p, stream, &launches,
                                    pl->profiling ? pl->events : nullptr);
    pl->launches = launches;
    if (pl->profiling && e == cudaSuccess) pl->profiled = true;
    if (e != cudaSuccess) return cuda_fail(e, "apply launch");
    return DEFMM_OK;
}

// Morton-contiguous split of the target leaves into nshards ranges of about
// equal estimated work: a leaf costs its near-field interactions plus, for
// every M2L pair of the leaf or an ancestor, 1.3 * N^3 (the measured cost of a
// pair relative to an interaction), shared among the ancestor's leaves by
// their points.  Returns the sorted-target range [t0, t1) of shard `shard`.
void shard_range(const HostPlan& hp, int nshards, int shard, int64_t* t0, int64_t* t1) {
    const Tree& tt = hp.tt;
    std::vector<int32_t> leaves;
    for (int32_t c = 0; c < tt.ncell(); ++c)
        if (tt.leaf(c) && tt.end[c] > tt.begin[c]) leaves.push_back(c);
    std::sort(leaves.begin(), leaves.end(), [&](int32_t a, int32_t b) { return tt.begin[a] < tt.begin[b]; });
    std::vector<double> pairs(tt.ncell(), 0.0);
    for (const auto& r : hp.m2l) pairs[r[0]] += 1.0;
    std::vector<double> cost(tt.ncell(), 0.0);   // per leaf cell
    for (size_t u = 0; u + 1 < hp.p2p_unit_off.size(); ++u) {
        const int32_t leaf = hp.p2p_leaf[hp.p2p_unit_leaf[u]];
        double ns = 0;
        for (int32_t k = hp.p2p_unit_off[u]; k < hp.p2p_unit_off[u + 1]; ++k) ns += hp.p2p_send[k] - hp.p2p_sbeg[k];
        cost[leaf] += ns * (double)(tt.end[leaf] - tt.begin[leaf]);
    }
    const double w = 1.3 * hp.NF;
    for (int32_t leaf : leaves) {
        const double np = (double)(tt.end[leaf] - tt.begin[leaf]);
        for (int32_t a = leaf; a >= 0; a = tt.parent[a])
            if (pairs[a] > 0) cost[leaf] += w * pairs[a] * np / (double)(tt.end[a] - tt.begin[a]);
    }
    double total = 0;
    for (int32_t leaf : leaves) total += cost[leaf];
    // boundary k: the first leaf whose preceding work reaches k * total / nshards
    auto boundary = [&](int k) -> int64_t {
        if (k <= 0) return 0;
        if (k >= nshards) return hp.nx;
        const double goal = total * k / nshards;
        double acc = 0;
        for (int32_t leaf : leaves) {
            if (acc >= goal) return tt.begin[leaf];
            acc += cost[leaf];
        }
        return hp.nx;
    };
    *t0 = boundary(shard);
    *t1 = std::max(*t0, boundary(shard + 1));
}

// Device lists of the shard: target cells overlapping [t0, t1) (a leaf of the
// shard or an ancestor of one) select the M2L groups and half-groups with such
// a member, the L2L entries of such sons, the L2P leaves, the P2P units and
// leaves.  Everything upward of M2L (P2M, M2M, M2F) stays whole.
defmm_status build_shard(defmm_plan_s* pl, int nshards, int shard, cudaStream_t stream) {
    const HostPlan& hp = pl->hp;
    auto& h = pl->sh;
    cudaFree(h.arena);
    h = defmm_plan_s::Shard();
    h.nshards = nshards;
    h.shard = shard;
    if (nshards == 1) return DEFMM_OK;
    shard_range(hp, nshards, shard, &h.t0, &h.t1);
    const Tree& tt = hp.tt;
    auto needed = [&](int32_t c) { return tt.begin[c] < h.t1 && tt.end[c] > h.t0; };
    std::vector<int32_t> grp, half, unit, leaf, l2p, big, small, mid, large;
    const size_t ngrp = hp.grp_member_off.size() - 1;
    for (size_t g = 0; g < ngrp; ++g)
        for (int32_t m = hp.grp_member_off[g]; m < hp.grp_member_off[g + 1]; ++m)
            if (needed(hp.l_cell[hp.grp_members[m]])) {
                grp.push_back((int32_t)g);
                const int nm = hp.grp_member_off[g + 1] - hp.grp_member_off[g];
                if (nm > 4) big.push_back((int32_t)g);
                else small.push_back((int32_t)(2 * g));
                if (nm > 7) large.push_back((int32_t)g);
                else if (nm > 4) mid.push_back((int32_t)g);
                break;
            }
    for (int32_t code : hp.grp_half) {
        const int32_t g = code >> 1, b = hp.grp_member_off[g] + 4 * (code & 1);
        const int32_t e = std::min(b + 4, hp.grp_member_off[g + 1]);
        for (int32_t m = b; m < e; ++m)
            if (needed(hp.l_cell[hp.grp_members[m]])) { half.push_back(code); break; }
    }
    for (size_t u = 0; u < hp.p2p_unit_leaf.size(); ++u)
        if (needed(hp.p2p_leaf[hp.p2p_unit_leaf[u]])) unit.push_back((int32_t)u);
    for (size_t li = 0; li < hp.p2p_leaf.size(); ++li)
        if (needed(hp.p2p_leaf[li])) leaf.push_back((int32_t)li);
    for (int32_t c : hp.l2p_cells)
        if (needed(c)) l2p.push_back(c);
    std::vector<std::vector<int32_t>> l2l(hp.l2l_lvl.size());
    for (size_t l = 0; l < hp.l2l_lvl.size(); ++l)
        for (size_t i = 0; i + 3 < hp.l2l_lvl[l].size(); i += 4)
            if (needed(hp.l_cell[hp.l2l_lvl[l][i]]))
                l2l[l].insert(l2l[l].end(), hp.l2l_lvl[l].begin() + i, hp.l2l_lvl[l].begin() + i + 4);
    // one device allocation, 256-byte aligned pieces
    std::vector<const std::vector<int32_t>*> parts = {&grp, &half, &unit, &leaf, &l2p, &big, &small, &mid, &large};
    for (auto& v : l2l) parts.push_back(&v);
    std::vector<size_t> off;
    size_t total = 0;
    for (auto* v : parts) {
        off.push_back(total);
        total += (v->size() * sizeof(int32_t) + 255) / 256 * 256;
    }
    if (total == 0) total = 256;
    std::vector<unsigned char> host(total, 0);
    for (size_t i = 0; i < parts.size(); ++i)
        if (!parts[i]->empty()) std::memcpy(host.data() + off[i], parts[i]->data(), parts[i]->size() * sizeof(int32_t));
    cudaError_t e = cudaMalloc(&h.arena, total);
    if (e == cudaSuccess) e = cudaMemcpyAsync(h.arena, host.data(), total, cudaMemcpyHostToDevice, stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(stream);
    if (e != cudaSuccess) {
        cudaFree(h.arena);
        h = defmm_plan_s::Shard();
        cudaGetLastError();
        return cuda_fail(e, "shard tables");
    }
    auto at = [&](size_t i) { return (const int32_t*)(h.arena + off[i]); };
    h.grp = at(0); h.n_grp = (int64_t)grp.size();
    h.half = at(1); h.n_half = (int64_t)half.size();
    h.unit = at(2); h.n_unit = (int64_t)unit.size();
    h.leaf = at(3); h.n_leaf = (int64_t)leaf.size();
    h.l2p = at(4); h.n_l2p = (int64_t)l2p.size();
    h.big = at(5); h.n_big = (int64_t)big.size();
    h.small = at(6); h.n_small = (int64_t)small.size();
    h.mid = at(7); h.n_mid = (int64_t)mid.size();
    h.large = at(8); h.n_large = (int64_t)large.size();
    h.l2l.resize(l2l.size());
    for (size_t l = 0; l < l2l.size(); ++l) h.l2l[l] = {at(9 + l), (int64_t)l2l[l].size() / 4};
    return DEFMM_OK;
}

}  // namespace

extern "C" {

defmm_status defmm_selftest_bounded_wait(int spins, void* stream) {
    if (spins < 1 || spins > (1 << 22)) return fail(DEFMM_ERR_ARG, "spins must be in [1, 2^22]");
    int* flag = nullptr;
    cudaError_t e = cudaMalloc(&flag, sizeof(int));
    if (e == cudaSuccess) e = cudaMemsetAsync(flag, 0, sizeof(int), (cudaStream_t)stream);
    if (e == cudaSuccess) e = launch_wait_probe(flag, spins, (cudaStream_t)stream);
    int h = 0;
    if (e == cudaSuccess) e = cudaMemcpyAsync(&h, flag, sizeof(int), cudaMemcpyDeviceToHost, (cudaStream_t)stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize((cudaStream_t)stream);
    cudaFree(flag);
    if (e != cudaSuccess) return cuda_fail(e, "bounded-wait self-test");
    return h ? fail(DEFMM_ERR_TIMEOUT, "device-side wait gave up (expected: nothing completes the phase)") : DEFMM_OK;
}

defmm_status defmm_plan_shard_range(defmm_plan plan, int nshards, int shard, int64_t* first, int64_t* count) {
    if (!plan || !first || !count) return fail(DEFMM_ERR_ARG, "plan, first and count must not be NULL");
    if (nshards < 1 || shard < 0 || shard >= nshards) return fail(DEFMM_ERR_ARG, "need 0 <= shard < nshards");
    int64_t t0 = 0, t1 = plan->hp.nx;
    if (nshards > 1) shard_range(plan->hp, nshards, shard, &t0, &t1);
    *first = t0;
    *count = t1 - t0;
    return DEFMM_OK;
}

defmm_status defmm_plan_set_shard(defmm_plan plan, int nshards, int shard, void* stream) {
    if (!plan) return fail(DEFMM_ERR_ARG, "plan is NULL");
    if (nshards < 1 || shard < 0 || shard >= nshards) return fail(DEFMM_ERR_ARG, "need 0 <= shard < nshards");
    if (plan->host_only) return fail(DEFMM_ERR_UNSUPPORTED, "plan was built with DEFMM_PLAN_HOST_ONLY");
    std::unique_lock<std::mutex> lk(plan->busy, std::try_to_lock);
    if (!lk.owns_lock()) return fail(DEFMM_ERR_BUSY, "plan is in use by another thread");
    // earlier applies may still read the old shard tables
    cudaError_t e = cudaStreamSynchronize((cudaStream_t)stream);
    if (e == cudaSuccess) e = cudaDeviceSynchronize();
    if (e != cudaSuccess) return cuda_fail(e, "set_shard synchronisation");
    return build_shard(plan, nshards, shard, (cudaStream_t)stream);
}

void defmm_default_options(defmm_options* opt) {
    if (!opt) return;
    opt->eta = 1.0;
    opt->hf_kw = 1.0;
    opt->fft_n = 0;
    opt->flags = 0;
    opt->self_eps = 1e-10;
    opt->hbm_budget = 0;
    opt->damping = 0.0;
    opt->radial_power = 1;
    opt->m2l_chunk_blocks = 0;
}

const char* defmm_last_error(void) { return g_err.c_str(); }

defmm_status defmm_plan_set_tuning(defmm_plan plan, const defmm_tuning* tuning) {
    if (!plan || !tuning) return fail(DEFMM_ERR_ARG, "plan or tuning is NULL");
    const int rb = tuning->m2l_rhs_block;
    if (rb != 0 && rb != 1 && rb != 2 && rb != 4) return fail(DEFMM_ERR_ARG, "m2l_rhs_block must be 0, 1, 2 or 4");
    if (tuning->p2p_tc_min_rhs < 0) return fail(DEFMM_ERR_ARG, "p2p_tc_min_rhs must be >= 0");
    if (tuning->p2p_reduce_phase != 0 && tuning->p2p_reduce_phase != 1)
        return fail(DEFMM_ERR_ARG, "p2p_reduce_phase must be 0 or 1");
    const int mb = tuning->m2l_members_per_block;
    if (mb != 0 && mb != 4 && mb != 8 && mb != 12 && mb != 14)
        return fail(DEFMM_ERR_ARG, "m2l_members_per_block must be 0, 4, 8, 12 or 14");
    std::lock_guard<std::mutex> g(plan->busy);
    plan->common.m2l_rb = rb;
    plan->common.p2p_tc_min_rhs = tuning->p2p_tc_min_rhs;
    plan->common.m2l_members = mb;
    plan->common.p2p_reduce_phase = tuning->p2p_reduce_phase;
    return DEFMM_OK;
}

defmm_status defmm_plan_get_tuning(defmm_plan plan, defmm_tuning* tuning) {
    if (!plan || !tuning) return fail(DEFMM_ERR_ARG, "plan or tuning is NULL");
    tuning->m2l_rhs_block = plan->common.m2l_rb;
    tuning->p2p_tc_min_rhs = plan->common.p2p_tc_min_rhs;
    tuning->m2l_members_per_block = plan->common.m2l_members;
    tuning->p2p_reduce_phase = plan->common.p2p_reduce_phase;
    return DEFMM_OK;
}

defmm_status defmm_plan_create(const double* X, int64_t nx, const double* Y, int64_t ny, double kappa, int order,
                               int leaf_size, const defmm_options* opt, void* stream, defmm_plan* out) {
    if (!out) return fail(DEFMM_ERR_ARG, "out is NULL");
    *out = nullptr;
    if (!X) return fail(DEFMM_ERR_ARG, "X is NULL");
    if (nx < 1) return fail(DEFMM_ERR_ARG, "nx must be >= 1");
    defmm_options o;
    defmm_default_options(&o);
    if (opt) o = *opt;
    bool same = (Y == nullptr) || (Y == X && ny == nx);
    if (!same && ny < 1) return fail(DEFMM_ERR_ARG, "ny must be >= 1");
    const bool host_only = (o.flags & DEFMM_PLAN_HOST_ONLY) != 0;
    if (!host_only) {
        std::call_once(g_config_once, [] {
            g_config_err = configure_kernels<float>();
            if (g_config_err == cudaSuccess) g_config_err = configure_kernels<double>();
        });
        if (g_config_err != cudaSuccess) return cuda_fail(g_config_err, "kernel configuration");
    }
    if (!(o.damping >= 0.0) || !std::isfinite(o.damping)) return fail(DEFMM_ERR_ARG, "damping must be finite and >= 0");
    if (o.radial_power != 1 && o.radial_power != 2) return fail(DEFMM_ERR_ARG, "radial_power must be 1 or 2");
    if (o.m2l_chunk_blocks < 0 || o.m2l_chunk_blocks == 1) return fail(DEFMM_ERR_ARG, "m2l_chunk_blocks must be 0 or >= 2");
    defmm_plan_s* pl = new (std::nothrow) defmm_plan_s;
    if (!pl) return fail(DEFMM_ERR_OOM, "host allocation");
    pl->hbm_budget = o.hbm_budget;
    std::vector<double> hx, hy;
    defmm_status s = read_points(X, nx, hx, host_only);
    if (s == DEFMM_OK && !same) s = read_points(Y, ny, hy, host_only);
    if (s != DEFMM_OK) { delete pl; return s; }
    try {
        // trees, traversal, directions and Alg. 2 marks on the device unless the plan is host-only
        const double* yp = same ? nullptr : hy.data();
        const int64_t nyy = same ? nx : ny;
        const auto t0 = std::chrono::steady_clock::now();
        double dev_ms = 0, front_ms = 0;
        FrontEnd front = [&](HostPlan& hp) {
            const auto f0 = std::chrono::steady_clock::now();
            device_front(hx.data(), nx, yp, nyy, leaf_size, hp, (cudaStream_t)stream, &dev_ms);
            front_ms = std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - f0).count();
        };
        build_host_plan(hx.data(), nx, yp, nyy, kappa, order, leaf_size, o.eta, o.hf_kw, o.fft_n, o.self_eps,
                        o.m2l_chunk_blocks, pl->hp, host_only ? nullptr : &front);
        const double all_ms = std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t0).count();
        pl->front_device_ms = dev_ms;
        pl->front_ms = front_ms;
        pl->host_ms = all_ms - front_ms;
    } catch (const std::bad_alloc&) {
        delete pl;
        return fail(DEFMM_ERR_OOM, "host allocation while building the plan");
    } catch (const DeviceFailure& ex) {
        delete pl;
        return fail(ex.out_of_memory ? DEFMM_ERR_OOM : DEFMM_ERR_CUDA, ex.what());
    } catch (const std::exception& ex) {
        delete pl;
        return fail(DEFMM_ERR_ARG, ex.what());
    }
    pl->hp.damping = o.damping;
    pl->hp.radial_power = o.radial_power;
    pl->host_only = host_only;
    {
        const auto u0 = std::chrono::steady_clock::now();
        s = host_only ? DEFMM_OK : upload(pl, hx, hy, (cudaStream_t)stream);
        pl->upload_ms = std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - u0).count();
    }
    if (s != DEFMM_OK) {
        cudaFree(pl->arena);
        delete pl;
        return s;
    }
    pl->X = std::move(hx);
    pl->Y = std::move(hy);
    *out = pl;
    return DEFMM_OK;
}

defmm_status defmm_plan_create_union(int ngeo, const double* const* X, const int64_t* nx, const double* kappa,
                                     int order, int leaf_size, const defmm_options* opt, void* stream,
                                     defmm_plan* out) {
    if (!out) return fail(DEFMM_ERR_ARG, "out is NULL");
    *out = nullptr;
    if (ngeo < 1 || !X || !nx || !kappa) return fail(DEFMM_ERR_ARG, "need ngeo >= 1 and X, nx, kappa arrays");
    for (int g = 0; g < ngeo; ++g) {
        if (!X[g] || nx[g] < 1) return fail(DEFMM_ERR_ARG, "every geometry needs points (X[g] != NULL, nx[g] >= 1)");
        if (!(kappa[g] >= 0.0) || !std::isfinite(kappa[g])) return fail(DEFMM_ERR_ARG, "kappa must be finite and >= 0");
    }
    defmm_options o;
    defmm_default_options(&o);
    if (opt) o = *opt;
    const bool host_only = (o.flags & DEFMM_PLAN_HOST_ONLY) != 0;
    if (!host_only) {
        std::call_once(g_config_once, [] {
            g_config_err = configure_kernels<float>();
            if (g_config_err == cudaSuccess) g_config_err = configure_kernels<double>();
        });
        if (g_config_err != cudaSuccess) return cuda_fail(g_config_err, "kernel configuration");
    }
    if (!(o.damping >= 0.0) || !std::isfinite(o.damping)) return fail(DEFMM_ERR_ARG, "damping must be finite and >= 0");
    if (o.radial_power != 1 && o.radial_power != 2) return fail(DEFMM_ERR_ARG, "radial_power must be 1 or 2");
    if (o.m2l_chunk_blocks < 0 || o.m2l_chunk_blocks == 1) return fail(DEFMM_ERR_ARG, "m2l_chunk_blocks must be 0 or >= 2");
    defmm_plan_s* pl = new (std::nothrow) defmm_plan_s;
    if (!pl) return fail(DEFMM_ERR_OOM, "host allocation");
    pl->hbm_budget = o.hbm_budget;
    std::vector<double> all;   // coordinates in the caller's order: geometry 0, then 1, ...
    try {
        std::vector<HostPlan> parts(ngeo);
        for (int g = 0; g < ngeo; ++g) {
            std::vector<double> hx;
            defmm_status s = read_points(X[g], nx[g], hx, host_only);
            if (s != DEFMM_OK) { delete pl; return s; }
            const double* xp = hx.data();
            const int64_t ng = nx[g];
            FrontEnd front = [&](HostPlan& hp) {
                double ms = 0;
                device_front(xp, ng, nullptr, ng, leaf_size, hp, (cudaStream_t)stream, &ms);
                pl->front_device_ms += ms;
            };
            build_host_plan(hx.data(), nx[g], nullptr, nx[g], kappa[g], order, leaf_size, o.eta, o.hf_kw, o.fft_n,
                            o.self_eps, o.m2l_chunk_blocks, parts[g], host_only ? nullptr : &front);
            parts[g].damping = o.damping;
            parts[g].radial_power = o.radial_power;
            all.insert(all.end(), hx.begin(), hx.end());
        }
        union_host_plans(parts, pl->hp);
    } catch (const std::bad_alloc&) {
        delete pl;
        return fail(DEFMM_ERR_OOM, "host allocation while building the plan");
    } catch (const DeviceFailure& ex) {
        delete pl;
        return fail(ex.out_of_memory ? DEFMM_ERR_OOM : DEFMM_ERR_CUDA, ex.what());
    } catch (const std::exception& ex) {
        delete pl;
        return fail(DEFMM_ERR_ARG, ex.what());
    }
    pl->host_only = host_only;
    defmm_status s = host_only ? DEFMM_OK : upload(pl, all, all, (cudaStream_t)stream);
    if (s != DEFMM_OK) {
        cudaFree(pl->arena);
        delete pl;
        return s;
    }
    pl->X = std::move(all);
    *out = pl;
    return DEFMM_OK;
}

defmm_status defmm_plan_save(defmm_plan plan, const char* path) {
    if (!plan || !path) return fail(DEFMM_ERR_ARG, "plan and path must not be NULL");
    try {
        save_plan_file(path, plan->hp, plan->X, plan->Y);
    } catch (const std::exception& ex) {
        return fail(DEFMM_ERR_ARG, ex.what());
    }
    return DEFMM_OK;
}

defmm_status defmm_plan_load(const char* path, const defmm_options* opt, void* stream, defmm_plan* out) {
    if (!out || !path) return fail(DEFMM_ERR_ARG, "path and out must not be NULL");
    *out = nullptr;
    defmm_options o;
    defmm_default_options(&o);
    if (opt) o = *opt;
    const bool host_only = (o.flags & DEFMM_PLAN_HOST_ONLY) != 0;
    if (!host_only) {
        std::call_once(g_config_once, [] {
            g_config_err = configure_kernels<float>();
            if (g_config_err == cudaSuccess) g_config_err = configure_kernels<double>();
        });
        if (g_config_err != cudaSuccess) return cuda_fail(g_config_err, "kernel configuration");
    }
    defmm_plan_s* pl = new (std::nothrow) defmm_plan_s;
    if (!pl) return fail(DEFMM_ERR_OOM, "host allocation");
    pl->hbm_budget = o.hbm_budget;
    try {
        load_plan_file(path, pl->hp, pl->X, pl->Y);
    } catch (const std::bad_alloc&) {
        delete pl;
        return fail(DEFMM_ERR_OOM, "host allocation while reading the plan file");
    } catch (const std::exception& ex) {
        delete pl;
        return fail(DEFMM_ERR_ARG, ex.what());
    }
    pl->host_only = host_only;
    defmm_status s = host_only ? DEFMM_OK : upload(pl, pl->X, pl->hp.same ? pl->X : pl->Y, (cudaStream_t)stream);
    if (s != DEFMM_OK) {
        cudaFree(pl->arena);
        delete pl;
        return s;
    }
    *out = pl;
    return DEFMM_OK;
}

defmm_status defmm_apply(defmm_plan plan, const void* q, void* p, int nrhs, defmm_dtype dtype, void* stream) {
    if (!plan) return fail(DEFMM_ERR_ARG, "plan is NULL");
    if (!q || !p) return fail(DEFMM_ERR_ARG, "q and p must be device pointers");
    if (nrhs < 1) return fail(DEFMM_ERR_ARG, "nrhs must be >= 1");
    if (dtype != DEFMM_C64 && dtype != DEFMM_C128) return fail(DEFMM_ERR_UNSUPPORTED, "dtype");
    if (plan->host_only) return fail(DEFMM_ERR_UNSUPPORTED, "plan was built with DEFMM_PLAN_HOST_ONLY");
    std::unique_lock<std::mutex> lk(plan->busy, std::try_to_lock);
    if (!lk.owns_lock()) return fail(DEFMM_ERR_BUSY, "plan is in use by another thread");
    if (dtype == DEFMM_C64) return apply_impl<float>(plan, plan->wf, q, p, nrhs, (cudaStream_t)stream);
    return apply_impl<double>(plan, plan->wd, q, p, nrhs, (cudaStream_t)stream);
}

defmm_status defmm_apply_slice(defmm_plan plan, const void* q, void* slice, int64_t ld, int nrhs, defmm_dtype dtype,
                               void* stream) {
    if (!plan) return fail(DEFMM_ERR_ARG, "plan is NULL");
    if (!q || !slice) return fail(DEFMM_ERR_ARG, "q and slice must be device pointers");
    if (nrhs < 1) return fail(DEFMM_ERR_ARG, "nrhs must be >= 1");
    if (dtype != DEFMM_C64 && dtype != DEFMM_C128) return fail(DEFMM_ERR_UNSUPPORTED, "dtype");
    if (plan->host_only) return fail(DEFMM_ERR_UNSUPPORTED, "plan was built with DEFMM_PLAN_HOST_ONLY");
    std::unique_lock<std::mutex> lk(plan->busy, std::try_to_lock);
    if (!lk.owns_lock()) return fail(DEFMM_ERR_BUSY, "plan is in use by another thread");
    const int64_t count = plan->sh.nshards > 1 ? plan->sh.t1 - plan->sh.t0 : plan->hp.nx;
    if (ld < count) return fail(DEFMM_ERR_ARG, "ld is smaller than the shard's target count");
    if (dtype == DEFMM_C64)
        return apply_impl<float>(plan, plan->wf, q, nullptr, nrhs, (cudaStream_t)stream, slice, ld);
    return apply_impl<double>(plan, plan->wd, q, nullptr, nrhs, (cudaStream_t)stream, slice, ld);
}

defmm_status defmm_assemble_slices(defmm_plan plan, int nshards, const int64_t* starts, const void* slices,
                                   int64_t ld, void* p, int nrhs, defmm_dtype dtype, void* stream) {
    if (!plan || !starts) return fail(DEFMM_ERR_ARG, "plan and starts must not be NULL");
    if (!slices || !p) return fail(DEFMM_ERR_ARG, "slices and p must be device pointers");
    if (nshards < 1 || nrhs < 1) return fail(DEFMM_ERR_ARG, "nshards and nrhs must be >= 1");
    if (dtype != DEFMM_C64 && dtype != DEFMM_C128) return fail(DEFMM_ERR_UNSUPPORTED, "dtype");
    if (plan->host_only) return fail(DEFMM_ERR_UNSUPPORTED, "plan was built with DEFMM_PLAN_HOST_ONLY");
    if (starts[0] != 0 || starts[nshards] != plan->hp.nx)
        return fail(DEFMM_ERR_ARG, "starts must run from 0 to the plan's target count");
    for (int s = 0; s < nshards; ++s) {
        if (starts[s + 1] < starts[s]) return fail(DEFMM_ERR_ARG, "starts must not decrease");
        if (starts[s + 1] - starts[s] > ld) return fail(DEFMM_ERR_ARG, "ld is smaller than a shard's target count");
    }
    const int esz = dtype == DEFMM_C64 ? 8 : 16;
    const char* src = static_cast<const char*>(slices);
    for (int s = 0; s < nshards; ++s) {
        cudaError_t e = launch_unslice(src + (size_t)s * nrhs * ld * esz, ld, p, plan->common.perm_t, plan->hp.nx, nrhs,
                                       starts[s], starts[s + 1], esz, plan->common.err_flag, (cudaStream_t)stream);
        if (e != cudaSuccess) return cuda_fail(e, "assemble slices");
    }
    return DEFMM_OK;
}

defmm_status defmm_apply_host(defmm_plan plan, const void* q_host, void* p_host, int nrhs, defmm_dtype dtype,
                              void* stream) {
    if (!plan) return fail(DEFMM_ERR_ARG, "plan is NULL");
    if (!q_host || !p_host) return fail(DEFMM_ERR_ARG, "q and p must be host pointers");
    if (nrhs < 1) return fail(DEFMM_ERR_ARG, "nrhs must be >= 1");
    if (dtype != DEFMM_C64 && dtype != DEFMM_C128) return fail(DEFMM_ERR_UNSUPPORTED, "dtype");
    if (plan->host_only) return fail(DEFMM_ERR_UNSUPPORTED, "plan was built with DEFMM_PLAN_HOST_ONLY");
    std::unique_lock<std::mutex> lk(plan->busy, std::try_to_lock);
    if (!lk.owns_lock()) return fail(DEFMM_ERR_BUSY, "plan is in use by another thread");
    cudaStream_t st = (cudaStream_t)stream;
    size_t csz = dtype == DEFMM_C64 ? sizeof(float2) : sizeof(double2);
    size_t qb = csz * (size_t)nrhs * plan->hp.ny, pb = csz * (size_t)nrhs * plan->hp.nx;
    defmm_status s;
    void *qd, *pd;
    if (dtype == DEFMM_C64) {
        s = ensure_workspace<float>(plan, plan->wf, nrhs, true);
        qd = plan->wf.q_stage; pd = plan->wf.p_stage;
    } else {
        s = ensure_workspace<double>(plan, plan->wd, nrhs, true);
        qd = plan->wd.q_stage; pd = plan->wd.p_stage;
    }
    if (s != DEFMM_OK) return s;
    CK(cudaMemcpyAsync(qd, q_host, qb, cudaMemcpyHostToDevice, st), "copy q to device");
    s = dtype == DEFMM_C64 ? apply_impl<float>(plan, plan->wf, qd, pd, nrhs, st)
                           : apply_impl<double>(plan, plan->wd, qd, pd, nrhs, st);
    if (s != DEFMM_OK) return s;
    CK(cudaMemcpyAsync(p_host, pd, pb, cudaMemcpyDeviceToHost, st), "copy p to host");
    CK(cudaStreamSynchronize(st), "apply");
    int flag[4] = {0, 0, 0, 0};
    CK(cudaMemcpy(flag, plan->common.err_flag, sizeof(flag), cudaMemcpyDeviceToHost), "read error flag");
    if (flag[0] == 2)
        return fail(DEFMM_ERR_CUDA, "a table index out of range (checked build; results invalid): kernels.cu line " +
                                        std::to_string(flag[1]) + ", index " + std::to_string(flag[2]) + ", size " +
                                        std::to_string(flag[3]));
    if (flag[0]) return fail(DEFMM_ERR_TIMEOUT, "a bounded device wait gave up (results invalid)");
    return DEFMM_OK;
}

defmm_status defmm_profile_enable(defmm_plan plan, int enable) {
    if (!plan) return fail(DEFMM_ERR_ARG, "plan is NULL");
    if (plan->host_only) return fail(DEFMM_ERR_UNSUPPORTED, "plan was built with DEFMM_PLAN_HOST_ONLY");
    if (enable && !plan->events[0])
        for (int i = 0; i <= kNumPhases; ++i) CK(cudaEventCreate(&plan->events[i]), "event create");
    plan->profiling = enable != 0;
    return DEFMM_OK;
}

defmm_status defmm_profile_read(defmm_plan plan, double* ms, int capacity, int* nphase) {
    if (!plan || !nphase) return fail(DEFMM_ERR_ARG, "null argument");
    if (!plan->profiled) return fail(DEFMM_ERR_ARG, "no profiled apply yet");
    CK(cudaEventSynchronize(plan->events[kNumPhases]), "profile wait");
    *nphase = kNumPhases;
    for (int i = 0; i < kNumPhases && i < capacity; ++i) {
        float t = 0.f;
        CK(cudaEventElapsedTime(&t, plan->events[i], plan->events[i + 1]), "profile elapsed");
        if (ms) ms[i] = (double)t;
    }
    return DEFMM_OK;
}

defmm_status defmm_destroy(defmm_plan plan) {
    if (!plan) return DEFMM_OK;
    if (plan->host_only) {
        delete plan;
        return DEFMM_OK;
    }
    cudaError_t e = cudaDeviceSynchronize();
    for (int i = 0; i <= kNumPhases; ++i)
        if (plan->events[i]) cudaEventDestroy(plan->events[i]);
    plan->wf.release();
    plan->wd.release();
    cudaFree(plan->arena);
    cudaFree(plan->sh.arena);
    delete plan;
    if (e != cudaSuccess) return cuda_fail(e, "destroy");
    return DEFMM_OK;
}

defmm_status defmm_plan_info(defmm_plan plan, defmm_info* out) {
    if (!plan || !out) return fail(DEFMM_ERR_ARG, "null argument");
    const HostPlan& hp = plan->hp;
    std::memset(out, 0, sizeof(*out));
    out->nx = hp.nx; out->ny = hp.ny; out->order = hp.p; out->fft_n = hp.N;
    out->nlevels = (int32_t)hp.tt.level_range.size();
    out->deepest_hf = hp.lv.l_hf;
    out->ncells_t = hp.tt.ncell(); out->ncells_s = hp.ts().ncell();
    out->n_m2l_pairs = (int64_t)hp.m2l.size(); out->n_p2p_pairs = (int64_t)hp.p2p.size();
    out->n_multipole = hp.nM(); out->n_local = hp.nL();
    out->n_fourier = (int64_t)hp.m2f_list.size();
    out->n_spectra = (int64_t)hp.spec_level.size();
    out->p2p_interactions = hp.p2p_interactions;
    out->plan_bytes = plan->arena_bytes;
    out->workspace_bytes = plan->wf.bytes + plan->wd.bytes;
    out->launches_per_apply = plan->launches;
    if (!plan->host_only) {
        int flag = 0;
        CK(cudaMemcpy(&flag, plan->common.err_flag, sizeof(int), cudaMemcpyDeviceToHost), "read error flag");
        out->device_error = flag;
    }
    out->d_aabb = hp.d_aabb;
    out->cube_side = hp.side;
    out->plan_front_device_ms = plan->front_device_ms;
    out->plan_front_ms = plan->front_ms;
    out->plan_host_ms = plan->host_ms;
    out->plan_upload_ms = plan->upload_ms;
    return DEFMM_OK;
}

defmm_status defmm_plan_table(defmm_plan plan, const char* name, int64_t* out, int64_t capacity, int64_t* count) {
    if (!plan || !name || !count) return fail(DEFMM_ERR_ARG, "null argument");
    const HostPlan& hp = plan->hp;
    std::vector<int64_t> v;
    std::string n(name);
    auto cells = [&](const Tree& t) {
        for (int32_t c = 0; c < t.ncell(); ++c) {
            int64_t row[7] = {t.level[c], t.ix[c], t.iy[c], t.iz[c], t.begin[c], t.end[c], t.parent[c]};
            v.insert(v.end(), row, row + 7);
        }
    };
    if (n == "perm_t") v.assign(hp.tt.perm.begin(), hp.tt.perm.end());
    else if (n == "perm_s") v.assign(hp.ts().perm.begin(), hp.ts().perm.end());
    else if (n == "cells_t") cells(hp.tt);
    else if (n == "cells_s") cells(hp.ts());
    else if (n == "m2l") for (auto& r : hp.m2l) v.insert(v.end(), {r[0], r[1], r[2]});
    else if (n == "p2p") for (auto& r : hp.p2p) v.insert(v.end(), {r[0], r[1]});
    else if (n == "mult") for (size_t e = 0; e < hp.m_cell.size(); ++e) v.insert(v.end(), {hp.m_cell[e], hp.m_dir[e]});
    else if (n == "local") for (size_t e = 0; e < hp.l_cell.size(); ++e) v.insert(v.end(), {hp.l_cell[e], hp.l_dir[e]});
    else if (n == "m2f_list") v.assign(hp.m2f_list.begin(), hp.m2f_list.end());
    else if (n == "spectra")
        for (size_t e = 0; e < hp.spec_level.size(); ++e)
            v.insert(v.end(), {hp.spec_level[e], hp.spec_kbar[e][0], hp.spec_kbar[e][1], hp.spec_kbar[e][2]});
    else if (n == "grp_member_off") v.assign(hp.grp_member_off.begin(), hp.grp_member_off.end());
    else if (n == "grp_members") v.assign(hp.grp_members.begin(), hp.grp_members.end());
    else if (n == "grp_chunk_off") v.assign(hp.grp_chunk_off.begin(), hp.grp_chunk_off.end());
    else if (n == "chk_blk_off") v.assign(hp.chk_blk_off.begin(), hp.chk_blk_off.end());
    else if (n == "chk_nspec") v.assign(hp.chk_nspec.begin(), hp.chk_nspec.end());
    else if (n == "chk_blk") v.assign(hp.chk_blk.begin(), hp.chk_blk.end());
    else if (n == "chk_op_off") v.assign(hp.chk_op_off.begin(), hp.chk_op_off.end());
    else if (n == "chk_op") v.assign(hp.chk_op.begin(), hp.chk_op.end());
    else if (n == "p2p_unit_leaf") v.assign(hp.p2p_unit_leaf.begin(), hp.p2p_unit_leaf.end());
    else if (n == "p2p_unit_off") v.assign(hp.p2p_unit_off.begin(), hp.p2p_unit_off.end());
    else if (n == "p2p_unit_ranges")
        for (size_t k = 0; k < hp.p2p_sbeg.size(); ++k) v.insert(v.end(), {hp.p2p_sbeg[k], hp.p2p_send[k]});
    else if (n == "p2p_leaf") v.assign(hp.p2p_leaf.begin(), hp.p2p_leaf.end());
    else return fail(DEFMM_ERR_ARG, "unknown table " + n);
    *count = (int64_t)v.size();
    if (out) std::memcpy(out, v.data(), sizeof(int64_t) * std::min<int64_t>(capacity, (int64_t)v.size()));
    return DEFMM_OK;
}

}  // extern "C"
