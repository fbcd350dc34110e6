// Discrete adjoint of the RK4 integration of Eq. 9.
#include "ftwa_internal.h"

namespace ftwa {

int launch_adjoint(Plan *, uint64_t, int64_t, int64_t, int32_t, const double *, double *, double *, double *,
                   cudaStream_t)
{
    return FTWA_ERR_UNSUPPORTED;
}

}  // namespace ftwa
