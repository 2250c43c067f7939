// Kernels for the basis size P = 1 and 1 quadrature node(s), FP32 and FP64.
#include "pgc_adjoint.cuh"
#include "pgc_batch.cuh"

namespace pgc {
Runner *make_runner_1x1(int precision, const HostTables &t, const DevBuffers &b, int num_sms)
{
    return make_runner_shape<1, 1>(precision, t, b, num_sms);
}
BatchRunner *make_batch_runner_1x1(int precision, const std::vector<BatchCase> &cases, const BatchScratch &sc,
                                    int num_sms)
{
    return make_batch_runner_shape<1, 1>(precision, cases, sc, num_sms);
}
size_t case_dev_size_1x1(int precision) { return case_dev_bytes<1, 1>(precision); }
AdjRunner *make_adj_runner_1x1(int precision, const HostTables &t, const DevBuffers &b, const AdjBuffers &ab,
                                int num_sms)
{
    return make_adj_runner_shape<1, 1>(precision, t, b, ab, num_sms);
}
}  // namespace pgc
