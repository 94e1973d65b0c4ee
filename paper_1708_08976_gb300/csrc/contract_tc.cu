// contract_tc.cu -- tensor-core (tcgen05) form of the contraction; see the kernel
// comments for the design.
#include "mtk_internal.cuh"

namespace mtk {

bool contract_tc_supported(const ContractParams& p, int precision) {
    (void)p; (void)precision;
    return false;
}

int contract_tc_i_tile(const ContractParams& p) {
    (void)p;
    return 128;
}

cudaError_t launch_contract_tc(const ContractParams& p, int precision, cudaStream_t s) {
    (void)p; (void)precision; (void)s;
    return cudaErrorNotSupported;
}

}  // namespace mtk
