// Temporary: the sequential batched launch.
#include "plan_internal.h"

poly_status ps_batched_impl(const poly_plan* plans, const void* const* fields, double* const* outs, int count,
                            cudaStream_t st) {
    for (int i = 0; i < count; i++) {
        poly_status s = poly_estimate(plans[i], fields[i], outs[i], nullptr, st);
        if (s != POLY_OK) return s;
    }
    return POLY_OK;
}
