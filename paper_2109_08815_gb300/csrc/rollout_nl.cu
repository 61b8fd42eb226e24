// Explicit instantiation of the rollout kernels for one chain length.  The
// build compiles this file once per link count (-DPDS_NL=1..8) so that the
// instantiations compile in parallel.
#include "rollout.cuh"

#ifndef PDS_NL
#error "compile with -DPDS_NL=<links>"
#endif

namespace pds {
template cudaError_t launch_rollout_nl<PDS_NL>(const ChainParams&, const float*, int, const Partials&, int, int32_t*,
                                               cudaStream_t, size_t, size_t);
template cudaError_t launch_simulate_nl<PDS_NL>(const ChainParams&, const float*, int, float*, cudaStream_t);
template int batch_rollout_blocks_per_sm_nl<PDS_NL>(int, int);
template cudaError_t launch_batch_rollout_nl<PDS_NL>(const BatchJob*, const WorkItem*, int, unsigned int*, int, int, int,
                                                     int, int, cudaStream_t);
}  // namespace pds
