// Tensor-core (tcgen05) implicit-GEMM convolution for the BF16 shading
// network.  Placeholder until the tcgen05 kernel lands: reports unsupported so
// that the CUDA-core kernel runs.
#include "internal.cuh"

namespace art {
struct ConvArgs;
bool tc_conv_supported(const ConvArgs&) { return false; }
void launch_tc_conv(art_ctx*, const ConvArgs&, const __nv_bfloat16*) {}
}  // namespace art
