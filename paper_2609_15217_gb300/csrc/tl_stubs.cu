// Entry points of the C ABI that are not in this translation unit yet.
#include "tinylu.h"
#include "tl_handle.h"

extern "C" {

tl_status tl_autotune(tl_handle *h, int, int, tl_layout, const char *)
{
    return h ? TL_ERR_UNSUPPORTED : TL_ERR_INVALID_ARG;
}

}
