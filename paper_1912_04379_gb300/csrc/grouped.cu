// Grouped SGEMM: planning and running many independent problems.
#include "internal.h"

extern "C" {

GB_API int gb_sgemm_grouped_plan(gb_handle_t, gb_algo_t, int64_t, const gb_gemm_problem_t *,
                                 gb_grouped_plan_t *plan, size_t *, int64_t *) {
    if (plan) *plan = nullptr;
    return GB_ERR_UNSUPPORTED;
}

GB_API int gb_sgemm_grouped_run(gb_grouped_plan_t, void *, size_t, void *) {
    return GB_ERR_PLAN;
}

GB_API int gb_sgemm_grouped_destroy(gb_grouped_plan_t plan) {
    return plan ? GB_ERR_PLAN : GB_OK;
}

}  // extern "C"
