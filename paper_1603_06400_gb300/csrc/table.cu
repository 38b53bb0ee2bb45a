// Table paths (exact piecewise-linear evaluation in u = sin(theta/2)).
#include "internal.cuh"

caxsi_status table_forward(caxsi_plan *, const float *, float *, int, cudaStream_t) {
    return CAXSI_ERR_UNSUPPORTED;
}
caxsi_status table_adjoint(caxsi_plan *, const float *, float *, int, cudaStream_t) {
    return CAXSI_ERR_UNSUPPORTED;
}
void table_destroy(caxsi_plan *) {}
