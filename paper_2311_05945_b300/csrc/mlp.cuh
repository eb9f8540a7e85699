// Small fully connected networks on the tensor cores (learned Newton warm
// start).  A network maps in[0] -> in[1] -> ... -> in[L] with ReLU after every
// layer but the last.  Weights are kept in FP32 (AdamW master copy) and used
// in BF16; products accumulate in FP32.
//
// Every product is one kernel, k_gemm_bf16: C = op(A) op(B) with BF16
// operands, warp-level mma.sync m16n8k16 tensor-core instructions and a
// fused epilogue (bias, ReLU, ReLU derivative).  The reductions over samples
// (weight and bias gradients, loss) are split over CTAs and summed in a
// fixed order, so training is bit-reproducible.
#pragma once
#include <cuda_bf16.h>

#include <vector>

#include "prims.cuh"

namespace zema {

using bf16 = __nv_bfloat16;

// Epilogues of k_gemm_bf16
enum GemmEpi : int {
    kEpiStore = 0,    // f32[z][m][n] = acc (z: split index)
    kEpiHidden = 1,   // z = acc + bias: f32 z, bf16 relu(z)
    kEpiOut = 2,      // f32 y = acc + bias
    kEpiReluBack = 3  // bf16 dz = acc * (z_in > 0)
};

struct GemmOut {
    float* f;          // f32 output (store / hidden pre-activation / out)
    bf16* h;           // bf16 output (hidden activation / back-propagated gradient)
    const float* bias; // per column
    const float* z_in; // pre-activation read by kEpiReluBack
    int ld;            // leading dimension of the outputs (= N)
};

struct Mlp {
    std::vector<int> dims;          // L + 1 layer widths
    std::vector<size_t> w_off, b_off;  // parameter offsets of W_l (in x out, row-major) and b_l
    size_t n_params = 0;
    cudaStream_t st = nullptr;
    Allocator A;
    DBuf<float> theta, grad, m, v, part;  // master weights, gradient, AdamW moments, split partials
    DBuf<bf16> theta_bf, theta_t, ones;  // BF16 weights; theta_t: each W_l transposed (out x in)
    // activations (for n rows): per hidden layer pre-activation (f32) and
    // activation (bf16), the input and output, two gradient buffers
    std::vector<DBuf<float>*> z;
    std::vector<DBuf<bf16>*> h;
    DBuf<bf16> xb, dy, dg0, dg1;
    DBuf<float> y, loss_part;
    int64_t cap_rows = 0;
    int64_t step = 0;
    int use_tc = 1;          // forward products on tcgen05 (0: warp-level mma.sync)
    DBuf<int> tc_err;        // set by a tcgen05 product whose completion wait timed out

    Mlp(const std::vector<int>& d, uint64_t seed, cudaStream_t s);
    ~Mlp();
    int layers() const { return (int)dims.size() - 1; }
    void ensure_rows(int64_t n);
    void refresh_bf16();
    void refresh_t();
    // y (n x out, f32, device) = net(x) for x (n x in, f32, device)
    void forward(const float* x, int64_t n, float* y_out);
    // MSE loss of net(x) against t, gradient into `grad`; returns the loss
    double backward(const float* x, const float* t, int64_t n);
    void adamw(float lr, float b1, float b2, float eps, float wd);
};

}  // namespace zema
