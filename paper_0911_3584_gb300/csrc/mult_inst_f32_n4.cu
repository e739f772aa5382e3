// Explicit instantiation of the block-product kernels for float, NSF=4.
#include "mult_kernels.cuh"

template lnv_status lnv::prod::dispatch_trans<float, 4>(lnv_ctx *, const lnv_plan *, const void *,
                                                      const void *, const void *, void *, void *);
