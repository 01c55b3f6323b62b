// Launchers not built yet.
#include "ot_internal.h"

namespace ota {

ot_status launch_solve_f64(ot_assoc_ctx* ctx, const SolveArgs64&, SolveSummary*) {
    return set_error(ctx, OT_EUNSUPPORTED, "FP64 solve not built");
}

ot_status launch_solve_lowp(ot_assoc_ctx* ctx, const SolveArgs&, int, double, SolveSummary*) {
    return set_error(ctx, OT_EUNSUPPORTED, "stored-kernel solve not built");
}

}  // namespace ota
