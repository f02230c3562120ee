// qsim_diff.cu -- reverse-mode gradients through the RK4 simulator (placeholder entry
// points; the adjoint kernels are added in the differentiation unit).
#include "qsim_internal.h"

using namespace qsim;

extern "C" size_t qsim_vjp_workspace(const qsim_vjp_desc* d) {
    (void)d;
    return 0;
}

extern "C" qsim_status qsim_rollout_vjp(const qsim_vjp_desc* d, const qsim_params* veh,
                                        const float* s0, const float* params, const float* actions,
                                        const float* actor, float* loss, float* g_actions,
                                        float* g_actor, float* g_params, float* actions_out,
                                        void* workspace, void* stream) {
    (void)d; (void)veh; (void)s0; (void)params; (void)actions; (void)actor; (void)loss;
    (void)g_actions; (void)g_actor; (void)g_params; (void)actions_out; (void)workspace; (void)stream;
    return fail(QSIM_ESTATE, "qsim_rollout_vjp: not available in this build");
}
