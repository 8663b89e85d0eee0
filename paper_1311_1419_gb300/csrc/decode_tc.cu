// K6: persistent tensor-core decode (tcgen05).  Not yet enabled: every shape
// reports unsupported and CS_ENGINE_AUTO selects the plain kernel.
#include "internal.h"

namespace csvc {

int tc_m_pad(int) { return 0; }
size_t tc_operand_bytes(int, int) { return 0; }
cudaError_t launch_prepare_tc(const float*, uint16_t*, int, int, int, cudaStream_t) {
    return cudaErrorNotSupported;
}
bool tc_supported(const cs_plan*, int) { return false; }
cudaError_t launch_decode_tc(const DecodeArgs&, cudaStream_t) { return cudaErrorNotSupported; }

}  // namespace csvc
