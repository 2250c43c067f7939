// Kernels for the basis size P = 1 and 1 quadrature node(s), FP32 and FP64.
#include "pgc_runner_impl.cuh"

namespace pgc {
Runner *make_runner_1x1(int precision, const HostTables &t, const DevBuffers &b, int num_sms)
{
    return make_runner_shape<1, 1>(precision, t, b, num_sms);
}
}  // namespace pgc
