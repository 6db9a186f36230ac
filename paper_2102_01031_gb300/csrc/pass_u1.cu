// pass_u1.cu -- fused drift + kick pass of the U(1) Abelian-Higgs model.
#include "common.cuh"

namespace clg {
typedef void (*PassKernel)(const PassArgs);
PassKernel u1_pass_kernel(int fp32, int red) { return nullptr; }
}  // namespace clg
