// mlp_tc.cu -- grouped matrix products of the atomic networks on the tensor
// cores (BF16 / FP16 operands, FP32 accumulation).
#include "nnp_internal.cuh"

namespace nnp {

bool tc_available() { return true; }

void launch_gemm_tc(const GemmProblem* probs, const GemmTile* tiles, int n_tiles, Prec p, int /*layer*/,
                    const void* /*maps*/, unsigned* /*status*/, cudaStream_t s) {
  launch_gemm_simt_typed(probs, tiles, n_tiles, p, s);
}

}  // namespace nnp
