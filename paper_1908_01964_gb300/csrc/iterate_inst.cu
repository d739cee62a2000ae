// One (BLOCK, SPT) shape of the accelerated kernels (see iterate.cu), selected by
// -DRCSCM_INST_BLOCK and -DRCSCM_INST_SPT at compile time.
#include "iterate_impl.cuh"

#if !defined(RCSCM_INST_BLOCK) || !defined(RCSCM_INST_SPT)
#error "compile with -DRCSCM_INST_BLOCK=<threads per row> -DRCSCM_INST_SPT=<slots per thread>"
#endif

namespace rcscm {
template cudaError_t launch_accel_t<RCSCM_INST_BLOCK, RCSCM_INST_SPT>(const DevState&, int, int, const IterParams&,
                                                                     bool, float2*, cudaStream_t);
}  // namespace rcscm
