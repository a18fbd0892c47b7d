// mp_errors.h -- bits of the per-mesh device error word.
#pragma once

namespace mp {
enum : int {
    DEV_ERR_NONFINITE = 1,  // the density held a NaN or an infinity
    DEV_ERR_TIMEOUT = 2,    // a bounded mbarrier wait gave up
    DEV_ERR_CONFIG = 4,     // a kernel was launched with an unusable configuration
};
}  // namespace mp
