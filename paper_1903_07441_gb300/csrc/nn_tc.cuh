// Host entry points of the tensor-memory convolution kernels (nn_conv_tc.cu)
// used by the network (nn_unet.cu).
#pragma once
#include <cuda_bf16.h>
#include <cuda_runtime.h>
#include <stddef.h>

namespace tw {
namespace nn {

typedef __nv_bfloat16 bf16;

// Every layer's tensor-core weights at once: entry l describes layer l (FP32
// weights at P + poff[l], cin[l] -> cout[l]); its forward arrangement goes to
// wf + foff[l], the arrangement of the transposed layer (cout -> cin, taps
// mirrored, for the data gradient) to wb + boff[l]; an offset of -1 skips one.
struct TcPrepTable {
    int n;
    long long poff[16], foff[16], boff[16];
    int cin[16], cout[16];
    long long total;   // sum over the layers of 2 cin cout 9 (forward and transposed slots)
};
int conv_tc_prepare_weights(const float *P, const TcPrepTable &t, bf16 *wf, bf16 *wb, cudaStream_t s);

bool conv3x3_tc_ok(int cin, int cout, int H, int W);
size_t conv3x3_tc_scratch_bytes(int cin, int cout);
int conv3x3_tc(const bf16 *X, const float *Wt, const float *b, const bf16 *S, bf16 *Y, int cin, int cout, int H,
               int W, int relu, void *scratch, cudaStream_t s, bool prearranged);
int conv3x3_tc_error(int *flag);
bool conv3x3_tc_narrow_ok(int cin, int cout, int H, int W);
int conv3x3_tc_narrow_splits(int cin, int cout, int H, int W, size_t part_floats);
int conv3x3_tc_narrow(const bf16 *X, const float *Wt, const float *b, const bf16 *S, bf16 *Y, int cin, int cout, int H,
                      int W, int relu, int splits, void *wscratch, float *part, cudaStream_t s, bool prearranged);
bool conv3x3_wgrad_tc_ok(int cin, int cout, int H, int W);
int conv3x3_wgrad_tc_plan(int cin, int cout, int H, int W, size_t cap_floats, int *chunk_px);
int conv3x3_wgrad_tc(const bf16 *X, const bf16 *dY, float *dW, float *db, int cin, int cout, int H, int W,
                     float *part, size_t part_floats, cudaStream_t s);

}  // namespace nn
}  // namespace tw
