// Instantiation of the tensor-core bound kernel for K = 16 kept noise
// symbols (Sec. 3.3 truncate); the device code is in tc_bound_impl.cuh.
#include "tc_bound_impl.cuh"

namespace sra {

template cudaError_t launch_tc_bound_kt<16>(int, bool, const TcParams &, const BoxSrc &, const BoundOut &, int,
                                            cudaStream_t);

}  // namespace sra
