// qsim_internal.h -- host-side handle layouts and error helpers shared by the library's
// translation units (not part of the public ABI).
#pragma once
#include <cuda_runtime.h>

#include <cstdint>

#include "../../include/qsim.h"
#include "qsim_device.cuh"

namespace qsim {

// Device pointers of an env set, passed by value to kernels.
struct EnvPtrs {
    float *state, *prm, *dist, *hist, *ep_ret, *ret_sum;
    uint32_t *ep_index, *ep_step, *n_done, *len_sum;
    float *rec, *side;
    int64_t rows;    // slots allocated in rec and side (the replay capacity)
    float* rewardC;  // [8]: C_rp C_rq C_rv C_rw C_ra C_rab C_rs, sigma_e
    int* status;
};

qsim_status fail(qsim_status s, const char* fmt, ...);
qsim_status cuda_fail(cudaError_t e, const char* what);
EnvCfg make_env_cfg(const qsim_config& c, const qsim_params& v, int n, int ld);
Vehicle make_vehicle(const qsim_params& v);

inline bool aligned16(const void* p) { return (reinterpret_cast<uintptr_t>(p) & 15u) == 0; }

}  // namespace qsim

#define QCHECK_CUDA(expr)                                                       \
    do {                                                                        \
        cudaError_t e_ = (expr);                                                \
        if (e_ != cudaSuccess) return qsim::cuda_fail(e_, #expr);               \
    } while (0)

#define QCHECK_LAUNCH(what)                                                     \
    do {                                                                        \
        cudaError_t e_ = cudaGetLastError();                                    \
        if (e_ != cudaSuccess) return qsim::cuda_fail(e_, what);                \
    } while (0)

struct qsim_handle {
    qsim_config cfg;
    qsim_params veh;
    qsim::EnvCfg dc;
    int device;
    int n, ld;
    int64_t capacity, t_now, head, size;
    int64_t next_curriculum;  // interaction count of the next curriculum change
    qsim::EnvPtrs p;
    int rollout_warps;
    // rollout scheduling: env partitions on internal streams, launched in time chunks so
    // that one partition's next chunk fills SMs the other leaves idle
    int rollout_parts, rollout_chunk;
    int rollout_packed;  // rollout engine: -1 automatic, 0 SIMT, 1 SIMT paired FMA, 2 tensor cores
    cudaStream_t part_stream[4];
    cudaEvent_t ev_fork, ev_join[4];
    bool streams_ready;
    int* tc_sched;  // persistent tensor-core rollout: [next unit, done chunks per group]
};

struct ac_handle {
    ac_config cfg;
    int device;
    int obs_dim, critic_in, hidden, batch;
    int n_actor, n_critic;
    int64_t t_actor, t_critic, updates;
    float* base;  // one allocation: [actor, actor_t, c1, c1_t, c2, c2_t, m_a, v_a, m_c1, v_c1, m_c2, v_c2]
    float *actor, *actor_t, *c1, *c1_t, *c2, *c2_t;
    float *m_a, *v_a, *m_c1, *v_c1, *m_c2, *v_c2;
    float* stats;     // [4]
    void* cache;      // device workspace + host copy of its descriptor for single-run launches
    uint32_t* idx_log;  // optional [batch] device log of the latest update's replay indices
    int* status;
};
