// contract_tc_px3_mn.cu -- the tensor-core contraction kernel with 3 BF16 pieces per tensor
// entry and an MN-major tensor operand (mode 0), both staging paths, in a translation unit
// of its own so that the kernel variants compile in parallel.
#include "contract_tc_kernel.cuh"

namespace mtk {

template cudaError_t tc_launch<3, true, true>(const tcd::TcParams&, const CUtensorMap&, dim3, size_t,
                                               cudaStream_t);
template cudaError_t tc_launch<3, true, false>(const tcd::TcParams&, const CUtensorMap&, dim3, size_t,
                                               cudaStream_t);

}  // namespace mtk
