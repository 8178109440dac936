// Internal: the object behind a defmm_plan handle, shared by the C-ABI files.
#pragma once

#include <cuda_runtime.h>

#include <mutex>
#include <string>
#include <vector>

#include "defmm.h"
#include "kernels.cuh"
#include "plan.h"

namespace defmm {

template <typename T> struct Workspace {
    int R = 0;
    typename Cplx<T>::type *qs = nullptr, *ps = nullptr, *M = nullptr, *Mhat = nullptr, *L = nullptr, *part = nullptr;
    void* q_stage = nullptr;
    void* p_stage = nullptr;
    size_t bytes = 0;
    void release() {
        cudaFree(qs); cudaFree(ps); cudaFree(M); cudaFree(Mhat); cudaFree(L); cudaFree(part);
        cudaFree(q_stage); cudaFree(p_stage);
        *this = Workspace();
    }
};

// Records msg as this thread's defmm_last_error() and returns s.
defmm_status set_error(defmm_status s, const std::string& msg);

}  // namespace defmm

struct defmm_plan_s {
    defmm::HostPlan hp;
    unsigned char* arena = nullptr;
    size_t arena_bytes = 0;
    defmm::DevCommon common{};
    defmm::DevTyped<float> tf{};
    defmm::DevTyped<double> td{};
    std::vector<defmm::LevelList> m2m, l2l;
    std::vector<const int32_t*> l2l_par;
    defmm::Workspace<float> wf;
    defmm::Workspace<double> wd;
    size_t hbm_budget = 0;
    int64_t launches = 0;
    bool host_only = false;
    bool profiling = false;
    bool profiled = false;
    cudaEvent_t events[defmm::kNumPhases + 1] = {};
    std::mutex busy;
    std::vector<double> X, Y;   // the coordinates the plan was built from (caller order; for plan files)
    // plan creation timing (ms): the device front end (CUDA events; wall time
    // of the call), the rest of the host construction, the upload and spectra
    double front_device_ms = 0, front_ms = 0, host_ms = 0, upload_ms = 0;
    // the shard this plan's defmm_apply computes (nshards == 1: the whole operator)
    struct Shard {
        int nshards = 1, shard = 0;
        int64_t t0 = 0, t1 = 0;                    // sorted targets written
        unsigned char* arena = nullptr;            // device copies of the lists below
        const int32_t *grp = nullptr, *half = nullptr, *unit = nullptr, *leaf = nullptr, *l2p = nullptr;
        const int32_t *big = nullptr, *small = nullptr, *mid = nullptr, *large = nullptr;
        int64_t n_grp = 0, n_half = 0, n_unit = 0, n_leaf = 0, n_l2p = 0, n_big = 0, n_small = 0, n_mid = 0, n_large = 0;
        std::vector<defmm::LevelList> l2l;
    } sh;
};

namespace defmm {

// The device tables an apply of this plan launches with: the whole operator,
// or, after defmm_plan_set_shard with more than one shard, the shard's target
// groups, near-field units and leaves, L2P cells, L2L lists and target range.
// Every apply entry point (plan scratch, caller workspace, static scratch)
// goes through this, so all of them compute the same shard.
inline DevCommon apply_tables(const defmm_plan_s* pl, const LevelList** l2l) {
    DevCommon c = pl->common;
    *l2l = pl->l2l.data();
    if (pl->sh.nshards > 1) {
        const auto& h = pl->sh;
        c.sh_on = 1;
        c.sh_grp = h.grp; c.n_grp = h.n_grp;
        c.grp_half = h.half; c.n_grp_half = h.n_half;
        c.grp_big = h.big; c.n_grp_big = h.n_big;
        c.grp_small = h.small; c.n_grp_small = h.n_small;
        c.grp_mid = h.mid; c.n_grp_mid = h.n_mid;
        c.grp_large = h.large; c.n_grp_large = h.n_large;
        c.sh_unit = h.unit; c.n_p2p_units = h.n_unit;
        c.sh_leaf = h.leaf; c.n_p2p_leaf = h.n_leaf;
        c.l2p_cells = h.l2p; c.n_l2p = h.n_l2p;
        c.sh_t0 = h.t0; c.sh_t1 = h.t1;
        *l2l = h.l2l.data();
    }
    return c;
}

}  // namespace defmm
