// Stored-kernel solver instantiated for __nv_bfloat16 storage (the code is in k_lowp.cuh).
#include "k_lowp.cuh"

namespace ota {

ot_status lowp_solve_bf16(ot_assoc_ctx* ctx, const SolveArgs& a, double absorb_log2, SolveSummary* sum_host) {
    return lowp_solve_t<__nv_bfloat16>(ctx, a, absorb_log2, sum_host);
}

}  // namespace ota
