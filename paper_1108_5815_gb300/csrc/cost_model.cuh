// cost_model.cuh -- state of the learned cost model (one per device).
#pragma once

#include <cuda_fp16.h>

#include <vector>

#include "kernels.cuh"

namespace fmm {

// Training samples: x = (log2 n_t, log2 n_s, sep, p); t = (ln ns per P2P pair,
// ln ns per M2L pair); m = which of the two t values was measured.
struct Samples {
    std::vector<float> x, t, m;
    int64_t size() const { return (int64_t)m.size() / 2; }
};

struct CostModel {
    bool trained = false;
    // device: FP16 parameters read by the forward pass, FP32 master copy and Adam moments
    __half *w16 = nullptr;
    float *w32 = nullptr, *mom = nullptr, *vel = nullptr, *grad = nullptr;
    float *loss = nullptr, *inv_cnt = nullptr;
    int *step = nullptr;
    // device: batch and per-block partial gradients
    float *x = nullptr, *t = nullptr, *m = nullptr, *partial = nullptr, *loss_part = nullptr;
    int64_t cap = 0;
    Samples last;  // samples of the last training
    ~CostModel();
    void ensure(int64_t nsamples);
};

// Sets the parameters (FP32 values, rounded to FP16 for the forward copy) and
// resets the Adam state.
void model_set(CostModel &cm, const float *params, cudaStream_t st);
// Initial parameters: uniform in +-sqrt(6 / (fan_in + fan_out)) from a SplitMix64
// stream, zero biases except b3 = the mean target of each output.
std::vector<float> model_init(const Samples &s, uint64_t seed);
// Loss and gradient of the current parameters over a batch (no update).
void model_grad(CostModel &cm, const Samples &s, float *loss, float *grad, cudaStream_t st);
// Full-batch Adam for `steps` steps (one captured CUDA graph per step); returns
// the loss before the first and after the last step.
void model_train(CostModel &cm, const Samples &s, int steps, float lr, float &loss0, float &loss1,
                 cudaStream_t st);
// One Adam step (for tests); *loss = the loss before the step.
void model_adam_step(CostModel &cm, const Samples &s, float lr, float *loss, cudaStream_t st);
void model_predict(CostModel &cm, const float *x, int64_t n, float *y, cudaStream_t st);
void model_table(CostModel &cm, int p, double theta, uint8_t *sel, cudaStream_t st);

// Artificial uniform particles in the unit cube, charges in [-1, 1) (SplitMix64).
void synth_uniform(float *xyz, float *q, int64_t n, uint64_t seed, cudaStream_t st);
// n points of a Plummer sphere (scale 1, radius <= 20), charges 1/n.
void synth_plummer(float *xyz, float *q, int64_t n, uint64_t seed, cudaStream_t st);

// Host-side SplitMix64 (Steele, Lea & Flood 2014) for sample features.
struct SplitMix64 {
    uint64_t s;
    uint64_t next()
    {
        uint64_t z = (s += 0x9e3779b97f4a7c15ull);
        z = (z ^ (z >> 30)) * 0xbf58476d1ce4e5b9ull;
        z = (z ^ (z >> 27)) * 0x94d049bb133111ebull;
        return z ^ (z >> 31);
    }
    double uniform() { return (double)(next() >> 11) * (1.0 / 9007199254740992.0); }
};

}  // namespace fmm
