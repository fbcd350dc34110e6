// BF16x3 connected Gram on the tcgen05 tensor cores.
#include "ftwa_internal.h"

namespace ftwa {

int launch_gram_bf16x3(Plan *, const void *, int64_t, int32_t, const double *, double *, double *, cudaStream_t)
{
    return FTWA_ERR_UNSUPPORTED;
}

}  // namespace ftwa
