// mlp.cu -- placeholder until the MLP occupancy kernels land.
#include "mlp.h"

namespace odc {
struct MlpState {};
odc_status mlp_check(const odc_mlp*, std::string* err) { *err = "MLP sources not built yet"; return ODC_ERR_UNSUPPORTED; }
odc_status mlp_prepare(MlpState**, const odc_mlp*, cudaStream_t, std::string* err) { *err = "MLP"; return ODC_ERR_UNSUPPORTED; }
void mlp_destroy(MlpState*) {}
odc_status mlp_grid(MlpState*, const GridDev&, float, uint32_t*, cudaStream_t, int64_t*, int64_t*, std::string*) { return ODC_ERR_UNSUPPORTED; }
odc_status mlp_bisect(MlpState*, const GridDev&, const uint32_t*, const uint32_t*, uint32_t, int, float, uint32_t*, cudaStream_t, int64_t*, int64_t*, std::string*) { return ODC_ERR_UNSUPPORTED; }
odc_status mlp_faces(MlpState*, const GridDev&, const uint32_t*, const uint32_t*, const WordInfo*, const uint32_t*, const uint32_t*, const uint32_t*, const uint8_t*, uint32_t, const SearchParams&, float, float2*, uint8_t*, cudaStream_t, int64_t*, int64_t*, std::string*) { return ODC_ERR_UNSUPPORTED; }
odc_status mlp_points(MlpState*, const float3*, int64_t, float, int, uint8_t*, float*, cudaStream_t, std::string*) { return ODC_ERR_UNSUPPORTED; }
}  // namespace odc
