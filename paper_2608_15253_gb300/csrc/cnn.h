// Host interface of the surrogate network's kernels (cnn.cu), used by the
// surrogate orchestration (surrogate.cu).
#pragma once

#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include <cstdint>

namespace mm {

struct ConvArgs {
    const __nv_bfloat16* in;   // [B][H+4][W+4][CIN] (halo 2)
    const uint4* wpk;          // packed weights [25][CIN/8][COUTP][8 bf16]
    const float* bias;         // [COUTP] or null
    void* out;                 // bf16 [B][H+4][W+4][COUTP] or f32 [B][H][W][3] (final layer)
    const __nv_bfloat16* mask; // input-gradient mode: multiply by (mask > 0)
    float out_scale;           // final layer
    int H, W;
    int* err;                  // set to 1 when a bounded wait runs out
    int rows_per_run;          // row-streaming kernel: output rows per CTA (set by the launcher)
    long wait_limit;           // polls before a bounded wait gives up (0: the default, 2^24)
    int skip_mma;              // test mode: issue no MMA and no commit (the wait must run out)
};

cudaError_t cnn_conv(int layer, bool backward, const ConvArgs& a, int B, cudaStream_t s);
cudaError_t cnn_conv_simt(int layer, const ConvArgs& a, const __nv_bfloat16* wplain, int B, cudaStream_t s);
void cnn_pack(cudaStream_t s, const float* w, int cout, int cin, int CINP, int COUTP, int flip, __nv_bfloat16* out);
void cnn_plain(cudaStream_t s, const float* w, int cout, int cin, int CINP, int COUTP, __nv_bfloat16* out);
// Weight and bias gradients of one layer, added into dw [cout][cin][5][5]
// and db [cout].  path 0: tensor-core kernel (CX, CZ in {16, 32}, not both
// 16), partial sums per CTA in part (cnn_dweight_parts() x kWgPartFloats
// floats), then a fixed-order reduction; err as in ConvArgs.  path 1: the
// SIMT cross-check (FP32 atomics; part and err unused).
constexpr int kWgPartFloats = 25 * 32 * 32 + 32;
int cnn_dweight_parts();
cudaError_t cnn_dweight(cudaStream_t s, int path, const __nv_bfloat16* dz, int CZ, int cout, const __nv_bfloat16* x,
                        int CX, int cin, int B, int H, int W, float* part, int* err, float* dw, float* db);
void cnn_mse_grad(cudaStream_t s, const float* y, const float* t, int B, int H, int W, __nv_bfloat16* dy,
                  double* loss);
void cnn_adam(cudaStream_t s, float* p, const float* g, float* m, float* v, int n, float lr, int t);
void cnn_dm_to_input(cudaStream_t s, const float* m, const float* mref, int H, int W, float c_in, __nv_bfloat16* x);
void cnn_field_from_output(cudaStream_t s, const float* out, const float* href, long long N, float Ms, float* H);

}  // namespace mm
