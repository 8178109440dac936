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
