// Kernels for the basis size P = 6 and 6 quadrature node(s), FP32 and FP64.
#include "pgc_runner_impl.cuh"

namespace pgc {
Runner *make_runner_6x6(int precision, const HostTables &t, const DevBuffers &b, int num_sms)
{
    return make_runner_shape<6, 6>(precision, t, b, num_sms);
}
}  // namespace pgc
