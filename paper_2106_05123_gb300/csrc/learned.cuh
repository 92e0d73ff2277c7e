// Learned CDF proposal for float32 keys: a tiny monotone model maps keys straight to buckets in
// place of the first sampled-splitter pass; every bucket that comes out larger than the base
// capacity is re-partitioned exactly by the splitter path.
//
// Model (a 2-layer MLP of width 16 with a hard-sigmoid hidden layer):
//   F(x) = sum_j a_j * sat(w_j * (xn - c_j)),  xn = (x - mu) / sigma,
//   a = softmax(alpha) (a_j > 0, sum 1), w_j = exp(omega_j) > 0, sat(z) = min(max(z, 0), 1).
// Each hidden unit is a ramp that starts at c_j with slope w_j; writing it as slope times the
// distance from its start keeps steep ramps (narrow clusters) well conditioned in float32.
// F is non-decreasing in x, and so is its float32 evaluation: every step (subtraction of a
// constant, product with a positive weight and saturation, fma-accumulate with a positive
// weight, scaling, truncation) is a correctly rounded monotone operation.  The bucket of x is min(nb - 1, trunc(nb * F(x))); NaNs go to the
// first (negative sign) or last bucket, so buckets are ordered by IEEE totalOrder and the
// result is exact whatever the model's quality; quality only changes bucket balance.
//
// Training: on a sorted sample xs[0..m) the target of xs[i] is its empirical CDF (i + 0.5) / m;
// the loss is the mean squared error, minimised with Adam over minibatches drawn from the whole
// sample, with the hand-written gradient below, by one cooperative launch of one CTA per SM.  Adam moves each ramp start in
// units of that ramp's initial width (c_j = c0_j + s_j d_j, d_j trained), so a step shifts a
// narrow ramp by a fraction of its own width rather than of the whole key range.
#pragma once

#include "kernels.cuh"

namespace pdq {

constexpr int kHidden = 16;
constexpr int kLearnedBuckets = 4096;
constexpr int kParams = 3 * kHidden;  // alpha[16], omega[16], beta[16]

// Inference form: normalisation folded in, h_j = sat(w_j * (x - t_j)) with t_j = mu + sigma c_j
// and w_j = exp(omega_j) / sigma.
struct LearnedModel {
  float w[kHidden], t[kHidden], a[kHidden];
  int nbuckets;
  int pad[3];
};

__device__ __forceinline__ int model_bucket(uint32_t code, const LearnedModel& m) {
  const uint32_t bits = Key<PDQ_F32>::dec(code);
  const int last = m.nbuckets - 1;
  if ((bits & 0x7FFFFFFFu) > 0x7F800000u) return (bits >> 31) ? 0 : last;  // NaN: by sign
  const float x = __uint_as_float(bits);
  float F = 0.f;
#pragma unroll
  for (int j = 0; j < kHidden; ++j) F = fmaf(m.a[j], __saturatef(m.w[j] * (x - m.t[j])), F);
  const int b = (int)(F * (float)m.nbuckets);
  return b < last ? b : last;
}

// Classifier policy over the learned model (float32 keys only; no equality bins).
struct ModelCls {
  static constexpr int kMaxBins = kLearnedBuckets;
  static constexpr bool kEqualBins = false;
  using Params = LearnedModel;
  struct Shared {
    int unused;
  };
  __device__ static int setup(Shared&, const Params& p, int) { return p.nbuckets; }
  __device__ static int nbins(const Params& p, int) { return p.nbuckets; }
  struct Classifier {
    const LearnedModel& m;
    __device__ __forceinline__ int operator()(uint32_t code) const { return model_bucket(code, m); }
    template <int N>
    __device__ __forceinline__ void vec(const uint32_t (&code)[N], int (&bin)[N]) const {
#pragma unroll
      for (int i = 0; i < N; ++i) bin[i] = model_bucket(code[i], m);
    }
  };
  template <class F>
  __device__ static void with(const Shared&, const Params& p, F&& f) {
    f(Classifier{p});
  }
};

// ------------------------------------------------------------------ training
// Parameter vector theta = [alpha(16), omega(16), c(16)] plus normalisation (mu, sigma).
struct TrainOut {
  float theta[kParams];
  float mu, sigma;
  float loss_first, loss_last;  // minibatch loss of the first and last step
  LearnedModel model;
  int status;                   // 0: trained; 1: a grid barrier gave up (model = last update)
  int pad[3];
};

// Forward of one point in the training parametrisation; fills h (hidden outputs), z (ramp
// inputs), a (softmax weights) and returns F.
__device__ __forceinline__ float model_forward(const float* theta, float xn, float* a, float* z, float* h) {
  float amax = theta[0];
#pragma unroll
  for (int j = 1; j < kHidden; ++j) amax = fmaxf(amax, theta[j]);
  float asum = 0.f;
#pragma unroll
  for (int j = 0; j < kHidden; ++j) {
    a[j] = __expf(theta[j] - amax);
    asum += a[j];
  }
  float F = 0.f;
#pragma unroll
  for (int j = 0; j < kHidden; ++j) {
    a[j] /= asum;
    z[j] = __expf(theta[kHidden + j]) * (xn - theta[2 * kHidden + j]);
    h[j] = fminf(fmaxf(z[j], 0.f), 1.f);
    F += a[j] * h[j];
  }
  return F;
}

// Gradient of 0.5 * (F - r)^2 with respect to theta for one point, accumulated into g.
__device__ __forceinline__ float model_point_grad(const float* theta, float xn, float r, float* g) {
  float a[kHidden], z[kHidden], h[kHidden];
  const float F = model_forward(theta, xn, a, z, h);
  const float e = F - r;
#pragma unroll
  for (int j = 0; j < kHidden; ++j) {
    const float inside = (z[j] > 0.f && z[j] < 1.f) ? 1.f : 0.f;  // derivative of sat
    const float w = __expf(theta[kHidden + j]);
    g[j] += e * a[j] * (h[j] - F);                                   // d/d alpha_j (softmax)
    g[kHidden + j] += e * a[j] * inside * (xn - theta[2 * kHidden + j]) * w;  // d/d omega_j
    g[2 * kHidden + j] -= e * a[j] * inside * w;                     // d/d c_j
  }
  return 0.5f * e * e;
}

// Same gradient with the per-step model terms precomputed: a (softmax weights), w (slopes) and c
// (ramp starts) in shared memory.
__device__ __forceinline__ float model_point_grad_pre(const float* a, const float* w, const float* c, float xn,
                                                      float r, float* g) {
  float h[kHidden];
  float F = 0.f;
#pragma unroll
  for (int j = 0; j < kHidden; ++j) {
    h[j] = fminf(fmaxf(w[j] * (xn - c[j]), 0.f), 1.f);
    F += a[j] * h[j];
  }
  const float e = F - r;
#pragma unroll
  for (int j = 0; j < kHidden; ++j) {
    const float z = w[j] * (xn - c[j]);
    const float ea = (z > 0.f && z < 1.f) ? e * a[j] : 0.f;
    g[j] += e * a[j] * (h[j] - F);
    g[kHidden + j] += ea * (xn - c[j]) * w[j];
    g[2 * kHidden + j] -= ea * w[j];
  }
  return 0.5f * e * e;
}

// Block sum of the kParams + 1 accumulators (gradient and loss); result in red[0..kParams].
template <int THREADS>
__device__ __forceinline__ void block_sum_params(float* g, float* red) {
  for (int i = threadIdx.x; i <= kParams; i += THREADS) red[i] = 0.f;
  __syncthreads();
#pragma unroll
  for (int i = 0; i <= kParams; ++i) {
    float v = g[i];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    if ((threadIdx.x & 31) == 0) atomicAdd(&red[i], v);
  }
  __syncthreads();
}

__device__ __forceinline__ bool finite_f(float x) { return (__float_as_uint(x) & 0x7F800000u) != 0x7F800000u; }

// Cross-CTA state of one training run (zeroed before the launch): gradient sums of three
// consecutive steps (rotating, so that a buffer is cleared two steps before it is refilled) and
// the grid barrier.
struct TrainSync {
  float gsum[3][kParams + 1];
  unsigned int count, gen, err, pad;
};

// Grid-wide barrier over all CTAs of a cooperative launch, bounded in time: false (for every
// thread of the CTA) when the other CTAs did not arrive within `limit_ns`.
__device__ __forceinline__ bool grid_barrier(TrainSync* sy, uint64_t limit_ns) {
  __shared__ int ok;
  __syncthreads();
  if (threadIdx.x == 0) {
    ok = 1;
    volatile unsigned int* vgen = &sy->gen;
    const unsigned int g = *vgen;  // cannot change before this CTA arrives
    __threadfence();
    if (atomicAdd(&sy->count, 1u) == gridDim.x - 1) {
      atomicExch(&sy->count, 0u);
      __threadfence();
      atomicAdd(&sy->gen, 1u);
    } else {
      const uint64_t t0 = global_ns();
      while (*vgen == g) {
        if (global_ns() - t0 > limit_ns) {
          ok = 0;
          atomicOr(&sy->err, 1u);
          break;
        }
        __nanosleep(64);
      }
    }
    __threadfence();
  }
  __syncthreads();
  return ok != 0;
}

// Training, one CTA per SM (cooperative launch): every CTA initialises the same parameters from
// the sample quantiles; per Adam step each CTA sums the gradient of its share of a minibatch of
// `batch` points of the sorted sample xs[0..m), the sums meet in global memory, and after a grid
// barrier every CTA applies the same Adam update to its own copy of the parameters (identical
// arithmetic on identical inputs keeps the copies equal).  CTA 0 writes the trained and folded
// model.
template <int THREADS>
__global__ void __launch_bounds__(THREADS)
learned_train_kernel(const float* __restrict__ xs, int64_t m, int steps, int batch, float lr, uint64_t seed,
                     TrainOut* out, TrainSync* sy) {
  __shared__ float theta[kParams], madam[kParams], vadam[kParams];
  __shared__ float c0[kHidden], cs[kHidden], dpos[kHidden];  // ramp start = c0 + cs * dpos
  __shared__ float pa[kHidden], pw[kHidden], pc[kHidden];    // this step's a, w, c
  __shared__ float red[kParams + 1];
  __shared__ float s_mu, s_sigma, s_loss;
  __shared__ int64_t s_lo, s_hi;  // finite range of the sorted sample
  const int tid = threadIdx.x;
  if (tid == 0) {
    int64_t lo = 0, hi = m;
    while (lo < hi && !finite_f(xs[lo])) ++lo;
    while (hi > lo && !finite_f(xs[hi - 1])) --hi;
    s_lo = lo;
    s_hi = hi;
    float mu = 0.f, sigma = 1.f;
    if (hi > lo) {
      mu = xs[lo + (hi - lo) / 2];
      const float span = xs[hi - 1] - xs[lo];
      sigma = span > 0.f ? span : 1.f;
    }
    s_mu = mu;
    s_sigma = sigma;
  }
  __syncthreads();
  const int64_t lo = s_lo, hi = s_hi;
  const float mu = s_mu, sigma = s_sigma;
  // initial ramps: ramp j rises across the j-th sixteenth of the finite sample
  for (int j = tid; j < kHidden; j += THREADS) {
    float q0 = 0.f, q1 = 1.f;
    if (hi > lo) {
      const int64_t n = hi - lo;
      q0 = (xs[lo + (n * j) / kHidden] - mu) / sigma;
      q1 = (xs[lo + (n * (j + 1) - 1) / kHidden] - mu) / sigma;
    }
    float width = q1 - q0;
    if (!(width > 1e-6f)) width = 1e-6f;
    theta[j] = 0.f;                     // equal weights
    theta[kHidden + j] = -logf(width);  // w = 1 / width: z = 1 at q1
    theta[2 * kHidden + j] = q0;        // the ramp starts at q0
    c0[j] = q0;
    cs[j] = width;
    dpos[j] = 0.f;
    madam[j] = madam[kHidden + j] = madam[2 * kHidden + j] = 0.f;
    vadam[j] = vadam[kHidden + j] = vadam[2 * kHidden + j] = 0.f;
  }
  __syncthreads();
  const float b1 = 0.9f, b2 = 0.999f, eps = 1e-8f;
  float loss_first = 0.f, loss_last = 0.f;
  bool ok = true;
  for (int step = 0; step < steps && hi > lo; ++step) {
    if (tid < kHidden) {
      float amax = theta[0];
      for (int j = 1; j < kHidden; ++j) amax = fmaxf(amax, theta[j]);
      float asum = 0.f;
      for (int j = 0; j < kHidden; ++j) asum += __expf(theta[j] - amax);
      pa[tid] = __expf(theta[tid] - amax) / asum;
      pw[tid] = __expf(theta[kHidden + tid]);
      pc[tid] = theta[2 * kHidden + tid];
    }
    __syncthreads();
    float g[kParams + 1];
#pragma unroll
    for (int i = 0; i <= kParams; ++i) g[i] = 0.f;
    for (int k = blockIdx.x * THREADS + tid; k < batch; k += gridDim.x * THREADS) {
      const uint64_t r = mix64(seed + ((uint64_t)step * (uint64_t)batch + (uint64_t)k + 1) * 0x9E3779B97F4A7C15ull);
      const int64_t i = lo + (int64_t)(r % (uint64_t)(hi - lo));
      const float target = ((float)i + 0.5f) / (float)m;
      g[kParams] += model_point_grad_pre(pa, pw, pc, (xs[i] - mu) / sigma, target, g);
    }
    block_sum_params<THREADS>(g, red);
    float* gs = sy->gsum[step % 3];
    if (tid <= kParams) atomicAdd(&gs[tid], red[tid]);
    if (!grid_barrier(sy, 1000000000ull)) {
      ok = false;
      break;
    }
    if (blockIdx.x == 0 && tid <= kParams) sy->gsum[(step + 2) % 3][tid] = 0.f;  // refilled at step + 2
    if (tid <= kParams) red[tid] = __ldcg(&gs[tid]);
    __syncthreads();
    if (tid < kParams) {
      const bool start = tid >= 2 * kHidden;  // ramp starts are trained in units of their width
      const int j = tid - 2 * kHidden;
      const float gi = red[tid] / (float)batch * (start ? cs[j] : 1.f);
      madam[tid] = b1 * madam[tid] + (1.f - b1) * gi;
      vadam[tid] = b2 * vadam[tid] + (1.f - b2) * gi * gi;
      const float mh = madam[tid] / (1.f - powf(b1, (float)(step + 1)));
      const float vh = vadam[tid] / (1.f - powf(b2, (float)(step + 1)));
      const float delta = lr * mh / (sqrtf(vh) + eps);
      if (start) {
        dpos[j] -= delta;
        theta[tid] = c0[j] + cs[j] * dpos[j];
      } else {
        theta[tid] -= delta;
      }
    }
    if (tid == 0) s_loss = red[kParams] / (float)batch;
    __syncthreads();
    if (step == 0) loss_first = s_loss;
    loss_last = s_loss;
  }
  if (blockIdx.x == 0 && tid == 0) {
    for (int i = 0; i < kParams; ++i) out->theta[i] = theta[i];
    out->mu = mu;
    out->sigma = sigma;
    out->loss_first = loss_first;
    out->loss_last = loss_last;
    out->status = ok ? 0 : 1;
    // fold: w' = w / sigma, t = mu + sigma c, a = softmax(alpha)
    float amax = theta[0];
    for (int j = 1; j < kHidden; ++j) amax = fmaxf(amax, theta[j]);
    float asum = 0.f;
    for (int j = 0; j < kHidden; ++j) asum += expf(theta[j] - amax);
    for (int j = 0; j < kHidden; ++j) {
      const float w = expf(theta[kHidden + j]) / sigma;
      out->model.w[j] = fmaxf(w, 1.17549435e-38f);  // strictly positive: monotone for +-inf too
      out->model.t[j] = mu + sigma * theta[2 * kHidden + j];
      out->model.a[j] = expf(theta[j] - amax) / asum;
    }
    out->model.nbuckets = kLearnedBuckets;
  }
}

constexpr int kTrainThreads = 256;

// Launches the training on one CTA per SM (cooperative launch: all CTAs are resident together,
// which the grid barrier needs).  `sy` must point at device memory for one TrainSync.
inline cudaError_t launch_learned_train(const float* xs, int64_t m, int steps, int batch, float lr, uint64_t seed,
                                        TrainOut* out, TrainSync* sy, int num_sms, cudaStream_t s) {
  cudaError_t e = cudaMemsetAsync(sy, 0, sizeof(TrainSync), s);
  if (e != cudaSuccess) return e;
  int per_sm = 0;
  e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, learned_train_kernel<kTrainThreads>, kTrainThreads, 0);
  if (e != cudaSuccess) return e;
  if (per_sm < 1) return cudaErrorCooperativeLaunchTooLarge;
  void* args[] = {(void*)&xs, (void*)&m, (void*)&steps, (void*)&batch, (void*)&lr, (void*)&seed, (void*)&out,
                  (void*)&sy};
  return cudaLaunchCooperativeKernel((const void*)learned_train_kernel<kTrainThreads>, dim3((unsigned)num_sms),
                                     dim3(kTrainThreads), args, 0, s);
}

// Full-batch loss and gradient (sums over the finite points, normalised by their count) at a
// given theta and normalisation: the probe the gradient-parity tests use.
template <int THREADS>
__global__ void __launch_bounds__(THREADS)
learned_grad_kernel(const float* __restrict__ xs, const float* __restrict__ targets, int64_t m,
                    const float* __restrict__ theta_g, float mu, float sigma, float* __restrict__ out) {
  __shared__ float theta[kParams];
  __shared__ float red[kParams + 1];
  for (int i = threadIdx.x; i < kParams; i += THREADS) theta[i] = theta_g[i];
  __syncthreads();
  float g[kParams + 1];
#pragma unroll
  for (int i = 0; i <= kParams; ++i) g[i] = 0.f;
  for (int64_t i = (int64_t)blockIdx.x * THREADS + threadIdx.x; i < m; i += (int64_t)gridDim.x * THREADS)
    g[kParams] += model_point_grad(theta, (xs[i] - mu) / sigma, targets[i], g);
  block_sum_params<THREADS>(g, red);
  for (int i = threadIdx.x; i <= kParams; i += THREADS) atomicAdd(&out[i], red[i]);
}

// Gathers m keys at hashed positions (the 1% training sample).
static __global__ void learned_gather_kernel(const float* __restrict__ keys, int64_t n, float* __restrict__ xs,
                                      int64_t m, uint64_t seed) {
  for (int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; j < m; j += (int64_t)gridDim.x * blockDim.x) {
    const uint64_t r = mix64(seed + (uint64_t)(j + 1) * 0x9E3779B97F4A7C15ull);
    xs[j] = keys[(int64_t)(r % (uint64_t)n)];
  }
}

}  // namespace pdq
