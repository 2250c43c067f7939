// Kernels for the basis size P = 21 and 36 quadrature node(s), FP32 and FP64.
#include "pgc_runner_impl.cuh"

namespace pgc {
Runner *make_runner_21x36(int precision, const HostTables &t, const DevBuffers &b, int num_sms)
{
    return make_runner_shape<21, 36>(precision, t, b, num_sms);
}
}  // namespace pgc
