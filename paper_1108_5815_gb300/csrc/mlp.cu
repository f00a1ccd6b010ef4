// mlp.cu -- the learned cost model's network: forward, backward, Adam and the
// selection-table inference, as CUDA kernels.
//
// The hybrid traversal chooses, for every pair the MAC accepts, the cheaper of
// cell-cell (M2L) and particle-particle (P2P) interaction (section "A new hybrid
// treecode-FMM with auto-tuning").  The paper times every kernel on artificial
// data and selects from those timings; here a small network is fitted to such
// timings and predicts the cost of one pair of either kind:
//     u  = (x - mu) / sd,   x = (log2 n_t, log2 n_s, sep, p)
//     h1 = tanh(W1 u + b1)  (64),  h2 = tanh(W2 h1 + b2)  (64)
//     y  = W3 h2 + b3,      y = (ln t_P2P, ln t_M2L), t in ns per pair
// Parameters are stored in FP16 (the copy the forward pass reads) with an FP32
// master copy for training; activations and sums are FP32.
// Loss over a batch with mask m: sum m (y - t)^2 / sum m.
#include <cuda_fp16.h>

#include "common.cuh"
#include "kernels.cuh"

namespace fmm {

namespace {

__device__ __forceinline__ void load_params(const __half *__restrict__ w16, float *sw, int tid, int nt)
{
    for (int i = tid; i < kMlpParams; i += nt) sw[i] = __half2float(w16[i]);
}

__device__ __forceinline__ void normalise(const float *x, float u[kMlpIn])
{
    const float mu[kMlpIn] = {5.f, 5.f, 3.f, 8.f};
    const float sd[kMlpIn] = {4.f, 4.f, 1.5f, 4.f};
#pragma unroll
    for (int i = 0; i < kMlpIn; ++i) u[i] = (x[i] - mu[i]) / sd[i];
}

// Forward pass of one sample with the parameters in shared memory.  h1 and h2
// (if not null) receive the hidden activations.
__device__ __forceinline__ void forward_one(const float *sw, const float u[kMlpIn], float *h1, float *h2,
                                            float y[kMlpOut])
{
    const float *W1 = sw + kOffW1, *b1 = sw + kOffB1, *W2 = sw + kOffW2, *b2 = sw + kOffB2,
                *W3 = sw + kOffW3, *b3 = sw + kOffB3;
    float a1[kMlpHidden];
#pragma unroll 8
    for (int j = 0; j < kMlpHidden; ++j) {
        float z = b1[j];
#pragma unroll
        for (int i = 0; i < kMlpIn; ++i) z = fmaf(W1[j * kMlpIn + i], u[i], z);
        a1[j] = tanhf(z);
        if (h1) h1[j] = a1[j];
    }
    float o0 = b3[0], o1 = b3[1];
    for (int j = 0; j < kMlpHidden; ++j) {
        float z = b2[j];
#pragma unroll 16
        for (int k = 0; k < kMlpHidden; ++k) z = fmaf(W2[j * kMlpHidden + k], a1[k], z);
        const float a2 = tanhf(z);
        if (h2) h2[j] = a2;
        o0 = fmaf(W3[j], a2, o0);
        o1 = fmaf(W3[kMlpHidden + j], a2, o1);
    }
    y[0] = o0;
    y[1] = o1;
}

constexpr int kGradSamples = 64;        // samples (= threads) per block of the gradient kernel
constexpr int kPad = kMlpHidden + 1;    // padded row of the per-sample activations

}  // namespace

size_t mlp_grad_smem()
{
    return sizeof(float) * ((size_t)kMlpParams + 4 * (size_t)kGradSamples * kPad +
                            (size_t)kGradSamples * (kMlpIn + kMlpOut) + kGradSamples);
}

// Predictions y[B][2] for features x[B][4].
__global__ void __launch_bounds__(128)
    k_mlp_forward(const __half *__restrict__ w16, const float *__restrict__ x, int B, float *__restrict__ y)
{
    __shared__ float sw[kMlpParams];
    load_params(w16, sw, threadIdx.x, blockDim.x);
    __syncthreads();
    const int s = blockIdx.x * blockDim.x + threadIdx.x;
    if (s >= B) return;
    float u[kMlpIn], o[kMlpOut];
    normalise(x + (int64_t)s * kMlpIn, u);
    forward_one(sw, u, nullptr, nullptr, o);
    y[(int64_t)s * 2] = o[0];
    y[(int64_t)s * 2 + 1] = o[1];
}

// Per-block partial gradient of the loss (samples blockIdx.x * 64 + threadIdx.x).
// inv_cnt = 1 / max(1, sum of the mask) over the whole batch.  partial[block][kMlpParams],
// loss_part[block] = sum over the block's samples of m (y - t)^2 * inv_cnt.
__global__ void __launch_bounds__(kGradSamples)
    k_mlp_grad_partial(const __half *__restrict__ w16, const float *__restrict__ x,
                       const float *__restrict__ t, const float *__restrict__ m, int B,
                       const float *__restrict__ inv_cnt_p, float *__restrict__ partial,
                       float *__restrict__ loss_part)
{
    extern __shared__ float smem[];
    float *sw = smem;
    float *sh1 = sw + kMlpParams;                 // [64][kPad]
    float *sh2 = sh1 + kGradSamples * kPad;
    float *sdz2 = sh2 + kGradSamples * kPad;
    float *sdz1 = sdz2 + kGradSamples * kPad;
    float *su = sdz1 + kGradSamples * kPad;       // [64][4]
    float *sdy = su + kGradSamples * kMlpIn;      // [64][2]
    float *sl = sdy + kGradSamples * kMlpOut;     // [64]
    const int tid = threadIdx.x;
    load_params(w16, sw, tid, blockDim.x);
    __syncthreads();
    const float inv_cnt = *inv_cnt_p;
    const int s = blockIdx.x * kGradSamples + tid;
    float *h1 = sh1 + tid * kPad, *h2 = sh2 + tid * kPad, *dz2 = sdz2 + tid * kPad, *dz1 = sdz1 + tid * kPad;
    if (s < B) {
        float u[kMlpIn], y[kMlpOut];
        normalise(x + (int64_t)s * kMlpIn, u);
        forward_one(sw, u, h1, h2, y);
        float l = 0.f;
        for (int k = 0; k < kMlpOut; ++k) {
            const float mk = m[(int64_t)s * 2 + k], e = y[k] - t[(int64_t)s * 2 + k];
            sdy[tid * 2 + k] = 2.f * mk * e * inv_cnt;
            l = fmaf(mk * e, e, l);
        }
        sl[tid] = l * inv_cnt;
        for (int i = 0; i < kMlpIn; ++i) su[tid * kMlpIn + i] = u[i];
        const float *W2 = sw + kOffW2, *W3 = sw + kOffW3;
        for (int j = 0; j < kMlpHidden; ++j)
            dz2[j] = (sdy[tid * 2] * W3[j] + sdy[tid * 2 + 1] * W3[kMlpHidden + j]) * (1.f - h2[j] * h2[j]);
        for (int i = 0; i < kMlpHidden; ++i) {
            float a = 0.f;
#pragma unroll 16
            for (int j = 0; j < kMlpHidden; ++j) a = fmaf(dz2[j], W2[j * kMlpHidden + i], a);
            dz1[i] = a * (1.f - h1[i] * h1[i]);
        }
    } else {
        for (int j = 0; j < kMlpHidden; ++j) h1[j] = h2[j] = dz2[j] = dz1[j] = 0.f;
        for (int i = 0; i < kMlpIn; ++i) su[tid * kMlpIn + i] = 0.f;
        sdy[tid * 2] = sdy[tid * 2 + 1] = 0.f;
        sl[tid] = 0.f;
    }
    __syncthreads();
    // thread r reduces over the block's samples: row r of W2 and W1, b1[r], b2[r], column r of W3
    float *g = partial + (int64_t)blockIdx.x * kMlpParams;
    const int r = tid;
    {
        float acc[kMlpHidden];
#pragma unroll
        for (int k = 0; k < kMlpHidden; ++k) acc[k] = 0.f;
        float db2 = 0.f, db1 = 0.f, w1[kMlpIn] = {0.f, 0.f, 0.f, 0.f}, w3a = 0.f, w3b = 0.f;
        for (int q = 0; q < kGradSamples; ++q) {
            const float d2 = sdz2[q * kPad + r], d1 = sdz1[q * kPad + r];
            const float *hq = sh1 + q * kPad;
#pragma unroll
            for (int k = 0; k < kMlpHidden; ++k) acc[k] = fmaf(d2, hq[k], acc[k]);
            db2 += d2;
            db1 += d1;
#pragma unroll
            for (int i = 0; i < kMlpIn; ++i) w1[i] = fmaf(d1, su[q * kMlpIn + i], w1[i]);
            const float a2 = sh2[q * kPad + r];
            w3a = fmaf(sdy[q * 2], a2, w3a);
            w3b = fmaf(sdy[q * 2 + 1], a2, w3b);
        }
#pragma unroll
        for (int k = 0; k < kMlpHidden; ++k) g[kOffW2 + r * kMlpHidden + k] = acc[k];
        g[kOffB2 + r] = db2;
        g[kOffB1 + r] = db1;
        for (int i = 0; i < kMlpIn; ++i) g[kOffW1 + r * kMlpIn + i] = w1[i];
        g[kOffW3 + r] = w3a;
        g[kOffW3 + kMlpHidden + r] = w3b;
    }
    if (tid < kMlpOut) {
        float db3 = 0.f;
        for (int q = 0; q < kGradSamples; ++q) db3 += sdy[q * 2 + tid];
        g[kOffB3 + tid] = db3;
    }
    if (tid == 0) {
        float l = 0.f;
        for (int q = 0; q < kGradSamples; ++q) l += sl[q];
        loss_part[blockIdx.x] = l;
    }
}

// inv_cnt = 1 / max(1, sum of the mask), one block.
__global__ void k_mlp_mask_count(const float *__restrict__ m, int n, float *__restrict__ inv_cnt)
{
    __shared__ float red[256];
    float a = 0.f;
    for (int i = threadIdx.x; i < n; i += blockDim.x) a += m[i];
    red[threadIdx.x] = a;
    __syncthreads();
    for (int o = blockDim.x / 2; o > 0; o >>= 1) {
        if (threadIdx.x < o) red[threadIdx.x] += red[threadIdx.x + o];
        __syncthreads();
    }
    if (threadIdx.x == 0) *inv_cnt = 1.f / fmaxf(red[0], 1.f);
}

// grad[i] = sum over blocks (in block order) of partial[b][i]; loss likewise.
__global__ void k_mlp_reduce(const float *__restrict__ partial, int nblk, const float *__restrict__ loss_part,
                             float *__restrict__ grad, float *__restrict__ loss)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < kMlpParams) {
        float a = 0.f;
        for (int b = 0; b < nblk; ++b) a += partial[(int64_t)b * kMlpParams + i];
        grad[i] = a;
    }
    if (i == 0) {
        float l = 0.f;
        for (int b = 0; b < nblk; ++b) l += loss_part[b];
        *loss = l;
    }
}

// Adam on the FP32 master weights (bias-corrected moments; step counter on the
// device so a captured graph can replay the step), then the FP16 copy.
__global__ void k_mlp_adam(float *__restrict__ w32, float *__restrict__ mom, float *__restrict__ vel,
                           const float *__restrict__ g, __half *__restrict__ w16, int *__restrict__ step,
                           float lr, float beta1, float beta2, float eps)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    const int t = *step + 1;
    if (i < kMlpParams) {
        const float mi = beta1 * mom[i] + (1.f - beta1) * g[i];
        const float vi = beta2 * vel[i] + (1.f - beta2) * g[i] * g[i];
        mom[i] = mi;
        vel[i] = vi;
        const float mh = mi / (1.f - powf(beta1, (float)t));
        const float vh = vi / (1.f - powf(beta2, (float)t));
        const float w = w32[i] - lr * mh / (sqrtf(vh) + eps);
        w32[i] = w;
        w16[i] = __float2half_rn(w);
    }
}

// The Adam step counter advances in a kernel of its own, after every block of
// k_mlp_adam has read it.
__global__ void k_mlp_step_inc(int *step) { *step += 1; }

// Selection table from the network: for every (target bucket, source bucket) the
// representative counts are the geometric means of the buckets' count ranges;
// sel = 1 (P2P) iff the predicted P2P time is below the predicted M2L time.
__global__ void __launch_bounds__(128)
    k_mlp_table(const __half *__restrict__ w16, float p, float sep, uint8_t *__restrict__ sel)
{
    __shared__ float sw[kMlpParams];
    load_params(w16, sw, threadIdx.x, blockDim.x);
    __syncthreads();
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= kSelNB * kSelNB) return;
    const int bt = i / kSelNB, bs = i % kSelNB;
    const float x[kMlpIn] = {bucket_mid_log2(bt), bucket_mid_log2(bs), sep, p};
    float u[kMlpIn], y[kMlpOut];
    normalise(x, u);
    forward_one(sw, u, nullptr, nullptr, y);
    sel[i] = y[0] < y[1] ? 1 : 0;
}

// Histogram of P2P pairs (target leaf, source cell) over the count buckets of
// the selection table: hist[bucket(n_t) * kSelNB + bucket(n_s)] (zeroed).
__global__ void k_pair_bucket_hist(const int *__restrict__ tgt, const int *__restrict__ src, int64_t n,
                                   const int *__restrict__ begin, const int *__restrict__ end,
                                   unsigned long long *__restrict__ hist)
{
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        const int t = tgt[i], so = src[i];
        atomicAdd(&hist[count_bucket(end[t] - begin[t]) * kSelNB + count_bucket(end[so] - begin[so])], 1ull);
    }
}

// The network's prediction of a solve's near- and far-field time: out[0] = sum
// over the occupied buckets of (pairs in the bucket) x exp(y_P2P) ns, out[1] =
// m2l_pairs x exp(y_M2L) ns (the M2L output does not depend on the counts; it
// is read at log2 counts 5, 5).  One block of kBlock threads.
__global__ void __launch_bounds__(256)
    k_mlp_solve_cost(const __half *__restrict__ w16, float p, float sep, const unsigned long long *__restrict__ hist,
                     unsigned long long m2l_pairs, double *__restrict__ out)
{
    __shared__ float sw[kMlpParams];
    __shared__ double part[256];
    load_params(w16, sw, threadIdx.x, blockDim.x);
    __syncthreads();
    double acc = 0.0;
    for (int i = threadIdx.x; i < kSelNB * kSelNB; i += blockDim.x) {
        const unsigned long long h = hist[i];
        if (h == 0) continue;
        const float x[kMlpIn] = {bucket_mid_log2(i / kSelNB), bucket_mid_log2(i % kSelNB), sep, p};
        float u[kMlpIn], y[kMlpOut];
        normalise(x, u);
        forward_one(sw, u, nullptr, nullptr, y);
        acc += (double)h * exp((double)y[0]);
    }
    part[threadIdx.x] = acc;
    __syncthreads();
    for (int s = blockDim.x / 2; s > 0; s >>= 1) {
        if ((int)threadIdx.x < s) part[threadIdx.x] += part[threadIdx.x + s];
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        const float x[kMlpIn] = {5.f, 5.f, sep, p};
        float u[kMlpIn], y[kMlpOut];
        normalise(x, u);
        forward_one(sw, u, nullptr, nullptr, y);
        out[0] = part[0];
        out[1] = (double)m2l_pairs * exp((double)y[1]);
    }
}

}  // namespace fmm
