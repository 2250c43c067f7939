// Kernels for one one-dimensional shape P = Q = PGC_1D_P (gPC degree M = P - 1 with M + 1 Gauss
// nodes), FP32 and FP64: the time-step kernels only.  The build compiles this unit once per entry
// of PGC_SHAPES_1D (pgc_runner.h) with -DPGC_1D_P=<P>.
#include "pgc_runner_impl.cuh"

#ifndef PGC_1D_P
#error "compile with -DPGC_1D_P=<basis size>"
#endif
#define PGC_CAT_(a, b) a##b
#define PGC_CAT(a, b) PGC_CAT_(a, b)

namespace pgc {
Runner *PGC_CAT(make_runner_1d_, PGC_1D_P)(int precision, const HostTables &t, const DevBuffers &b, int num_sms)
{
    return make_runner_shape<PGC_1D_P, PGC_1D_P>(precision, t, b, num_sms);
}
}  // namespace pgc
