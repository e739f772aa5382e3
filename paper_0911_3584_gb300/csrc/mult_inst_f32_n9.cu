// Explicit instantiation of the block-product kernels for float, NSF=9.
#include "mult_kernels.cuh"

template lnv_status lnv::prod::dispatch_trans<float, 9>(lnv_ctx *, const lnv_plan *, const void *,
                                                      const void *, const void *, void *, void *);
