// Explicit instantiation of the block-product kernels for double, NSF=1.
#include "mult_kernels.cuh"

template lnv_status lnv::prod::dispatch_trans<double, 1>(lnv_ctx *, const lnv_plan *, const void *,
                                                      const void *, const void *, void *, void *);
