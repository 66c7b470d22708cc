// Instantiation of the tensor-core bound kernel for K = 128 kept noise
// symbols (Sec. 3.3 truncate; widths 128 and 256, one box per tile); the
// device code is in tc_bound_impl.cuh.
#include "tc_bound_impl.cuh"

namespace sra {

template cudaError_t launch_tc_bound_kt<128>(int, bool, const TcParams &, const BoxSrc &, const BoundOut &, int,
                                             cudaStream_t);

}  // namespace sra
