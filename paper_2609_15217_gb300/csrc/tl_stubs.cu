// Entry points of the C ABI that are not in this translation unit yet.
#include "tinylu.h"
#include "tl_handle.h"

extern "C" {

tl_status tl_lupp_solve_batched(tl_handle *h, int64_t, const int32_t *, const int64_t *, const double *,
                                const int64_t *, const double *, double *, const int64_t *, int32_t *,
                                int32_t *, tl_precision, int32_t *, cudaStream_t)
{
    return h ? TL_ERR_UNSUPPORTED : TL_ERR_INVALID_ARG;
}

tl_status tl_autotune(tl_handle *h, int, int, tl_layout, const char *)
{
    return h ? TL_ERR_UNSUPPORTED : TL_ERR_INVALID_ARG;
}

}
