// mlp_tc.cu -- BF16 tensor-core (tcgen05) path of the MLP occupancy network.
#include "mlp.h"
#include "mlp_dev.cuh"

namespace odc {
struct MlpTc {};
odc_status mlp_tc_prepare(MlpState*, const float*, cudaStream_t, std::string*) { return ODC_OK; }
odc_status mlp_tc_eval(MlpState*, const float3*, const GridDev&, int64_t, float*, cudaStream_t, std::string* err) {
    *err = "BF16 path not built yet";
    return ODC_ERR_UNSUPPORTED;
}
void mlp_tc_destroy(MlpState*) {}
}  // namespace odc
