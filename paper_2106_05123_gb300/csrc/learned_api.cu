// C ABI test probes of the learned-CDF model (training and gradient); the learned sort itself
// is instantiated with the other float32 kernels (inst_f32.cu).
#include <cstring>
#include <string>

#include "sort_impl.cuh"

using namespace pdq;

extern "C" {

size_t pdq_workspace_bytes_learned(int64_t n) { return n < 0 ? 0 : learned_workspace_bytes(n); }

// Gradient probe: full-batch loss and gradient of the learned model's training objective.
int pdq_learned_loss_grad(const float* d_x, const float* d_targets, int64_t m, const float* h_theta,
                          float mu, float sigma, float* h_out, void* d_ws, void* cuda_stream) {
  if (m < 0 || !h_theta || !h_out || (m > 0 && (!d_x || !d_targets)) || !d_ws)
    return set_error(PDQ_ERR_ARG, "bad argument");
  cudaStream_t s = static_cast<cudaStream_t>(cuda_stream);
  float* d_theta = static_cast<float*>(d_ws);
  float* d_out = d_theta + kParams;
  cudaError_t e = cudaMemcpyAsync(d_theta, h_theta, sizeof(float) * kParams, cudaMemcpyHostToDevice, s);
  if (e == cudaSuccess) e = cudaMemsetAsync(d_out, 0, sizeof(float) * (kParams + 1), s);
  if (e != cudaSuccess) return set_error(PDQ_ERR_CUDA, cudaGetErrorString(e));
  if (m > 0) {
    LaunchScope ls("learned_grad", s, 0.0);
    const unsigned blocks = (unsigned)std::min<int64_t>((m + 255) / 256, 1024);
    learned_grad_kernel<256><<<blocks, 256, 0, s>>>(d_x, d_targets, m, d_theta, mu, sigma, d_out);
  }
  e = cudaGetLastError();
  if (e == cudaSuccess) e = cudaMemcpyAsync(h_out, d_out, sizeof(float) * (kParams + 1), cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  if (e != cudaSuccess) return set_error(PDQ_ERR_CUDA, cudaGetErrorString(e));
  return PDQ_OK;
}

// Training probe: trains the model on a sorted sample d_xs[0..m) and returns theta (48 floats),
// then mu, sigma, first-step loss, last-step loss (4 floats), and the folded model's w, t, a.
int pdq_learned_train(const float* d_xs, int64_t m, int steps, int batch, float lr, void* d_ws,
                      float* h_theta, float* h_norm_loss, float* h_wba, void* cuda_stream) {
  if (m <= 0 || !d_xs || !d_ws || steps < 0 || batch <= 0) return set_error(PDQ_ERR_ARG, "bad argument");
  cudaStream_t s = static_cast<cudaStream_t>(cuda_stream);
  TrainOut* d_out = static_cast<TrainOut*>(d_ws);
  TrainSync* d_sync = reinterpret_cast<TrainSync*>(static_cast<char*>(d_ws) + align_up(sizeof(TrainOut), 256));
  int dev = 0, sms = 0;
  cudaGetDevice(&dev);
  if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || sms <= 0) sms = 1;
  cudaError_t e;
  {
    LaunchScope ls("learned_train", s, 0.0);
    e = launch_learned_train(d_xs, m, steps, batch, lr, 0x7A11ull, d_out, d_sync, sms, s);
  }
  if (e != cudaSuccess) return set_error(PDQ_ERR_CUDA, std::string("learned_train: ") + cudaGetErrorString(e));
  TrainOut h;
  e = cudaGetLastError();
  if (e == cudaSuccess) e = cudaMemcpyAsync(&h, d_out, sizeof(h), cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  if (e != cudaSuccess) return set_error(PDQ_ERR_CUDA, cudaGetErrorString(e));
  if (h.status) return set_error(PDQ_ERR_TIMEOUT, "learned_train: a grid barrier gave up");
  if (h_theta) std::memcpy(h_theta, h.theta, sizeof(h.theta));
  if (h_norm_loss) {
    h_norm_loss[0] = h.mu;
    h_norm_loss[1] = h.sigma;
    h_norm_loss[2] = h.loss_first;
    h_norm_loss[3] = h.loss_last;
  }
  if (h_wba) {
    std::memcpy(h_wba, h.model.w, sizeof(h.model.w));
    std::memcpy(h_wba + kHidden, h.model.t, sizeof(h.model.t));
    std::memcpy(h_wba + 2 * kHidden, h.model.a, sizeof(h.model.a));
  }
  return PDQ_OK;
}

}  // extern "C"
