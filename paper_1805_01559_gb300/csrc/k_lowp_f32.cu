// Stored-kernel solver instantiated for float storage (the code is in k_lowp.cuh).
#include "k_lowp.cuh"

namespace ota {

ot_status lowp_solve_f32(ot_assoc_ctx* ctx, const SolveArgs& a, double absorb_log2, SolveSummary* sum_host) {
    return lowp_solve_t<float>(ctx, a, absorb_log2, sum_host);
}

}  // namespace ota
