// Per-iteration variant selection and the selector MLP.
//
// Before every iteration k the decide kernel picks how the frontier expansion
// runs: a full pull pass, a SlimWork pull pass, a compacted-frontier push, or a
// visited-filtered pull (all compute the same x_k).  Fixed policies always
// pick one; the heuristic policy switches between push and filtered pull on
// frontier size (top-down while the frontier's edges are few compared with
// the unexplored ones); the learned policy evaluates a 16-64-64-4 MLP on the
// iteration's features and takes the variant with the smallest predicted
// log-time, except for frontiers small enough for the cluster push, which both
// adaptive policies hand to it.  Schedules never change results, only their cost.
//
// MLP parameters (fp32, 5508 values, inputs first):
//   W1[16][64] | b1[64] | W2[64][64] | b2[64] | W3[64][4] | b3[4]
//   h1 = relu(x W1 + b1), h2 = relu(h1 W2 + b2), y = h2 W3 + b3.
#include <cmath>

#include "ss_device.cuh"

namespace ss {

constexpr int F_IN = SS_SELECTOR_FEATURES, F_H = SS_SELECTOR_HIDDEN, F_OUT = SS_SELECTOR_OUTPUTS;
constexpr int OFF_W1 = 0, OFF_B1 = OFF_W1 + F_IN * F_H, OFF_W2 = OFF_B1 + F_H,
              OFF_B2 = OFF_W2 + F_H * F_H, OFF_W3 = OFF_B2 + F_H, OFF_B3 = OFF_W3 + F_H * F_OUT,
              N_PARAMS = OFF_B3 + F_OUT;
static_assert(N_PARAMS == SS_SELECTOR_PARAMS, "selector parameter count");

constexpr int PUSH_UNIT_SEL = 256;  // must match the push kernels' unit size
constexpr int DECIDE_THREADS = 256;  // the decide block (the MLP uses its first F_H threads)
static_assert(N_PARAMS % 4 == 0, "weights are staged as float4");

// Frontier-size rule (top-down / bottom-up switching with alpha = 14, beta = 24).
__device__ int heuristic_variant(const Dev& d, const Ctl* c) {
  const unsigned long long nf = c->prev_new, mf = c->prev_deg;
  const unsigned long long mu = (unsigned long long)d.nnz - c->reached_deg;
  if (c->prev_variant < 0) return VAR_PUSH;
  // a frontier the cluster push takes is cheaper there than in any grid-wide pass
  if (local_fits(d, nf, mf)) return VAR_PUSH;
  if (c->prev_variant == VAR_PUSH || c->prev_variant == VAR_PUSH_LOCAL) return (14ull * mf > mu) ? VAR_FILTERED : VAR_PUSH;
  const bool shrinking = c->prev_new < c->prev2_new;
  return (24ull * nf < (unsigned long long)d.n && shrinking) ? VAR_PUSH : VAR_FILTERED;
}

__device__ __forceinline__ bool push_fits(const Dev& d, const Ctl* c) {
  const unsigned long long need = c->prev_new + c->prev_deg / PUSH_UNIT_SEL + 1;
  return need <= (unsigned long long)d.units_cap;
}

// One block of DECIDE_THREADS threads.  Writes ctl->variant and sets the switch.  In the
// device-side loop it also ends the loop (WHILE condition 0) if the run is
// already done or has looped more than n + 2 times, so termination never
// depends on a later kernel.
__global__ void __launch_bounds__(DECIDE_THREADS) k_decide(Dev d, int policy, cudaGraphConditionalHandle sw,
                                                            int use_sw, cudaGraphConditionalHandle cw,
                                                            int use_cw) {
  __shared__ float x[F_IN], h1[F_H], h2[F_H], y[F_OUT];
  __shared__ __align__(16) float wsh[N_PARAMS];  // the selector weights, staged once per decision
  __shared__ int choice, stop;
  Ctl* c = d.ctl;
  const int t = threadIdx.x;
  // a frontier the cluster push takes stays with it (that launch runs the
  // following small levels too, a saving no per-level time can express), so the
  // network is evaluated only on levels that need a grid-wide pass; elsewhere the
  // learned policy takes the frontier-size rule's choice, the cluster push
  const bool net = policy == SS_V_LEARNED && d.mlp != nullptr && !local_fits(d, c->prev_new, c->prev_deg);
  if (net)  // in flight while thread 0 computes the features
    for (int i = t; i < N_PARAMS / 4; i += DECIDE_THREADS)
      reinterpret_cast<float4*>(wsh)[i] = __ldg(reinterpret_cast<const float4*>(d.mlp) + i);
  if (t == 0) {
    stop = c->done;  // host-driven queued loops launch past the end of a run
    if (use_cw) {
      c->loop_guard += 1;
      if (c->done || c->loop_guard > (unsigned long long)d.n + 2) {
        if (!c->done) {
          c->error |= 4;
          c->done = 1;
        }
        stop = 1;
        cudaGraphSetConditional(cw, 0u);
        if (use_sw) cudaGraphSetConditional(sw, (unsigned)VAR_FULL);  // its kernels see done
      }
    }
  }
  __syncthreads();
  if (stop) return;
  if (t == 0) {
    compute_features(d, c, x);
    const int k = c->k;
    if (k < d.iter_cap)
      for (int i = 0; i < F_IN; ++i) d.feats[(size_t)k * F_IN + i] = x[i];
    int v;
    switch (policy) {
      case SS_V_FULL: v = VAR_FULL; break;
      case SS_V_SLIMWORK: v = VAR_SLIMWORK; break;
      case SS_V_PUSH: v = VAR_PUSH; break;
      case SS_V_PULL_FILTERED: v = VAR_FILTERED; break;
      default: v = heuristic_variant(d, c); break;
    }
    choice = v;
  }
  __syncthreads();
  if (net) {
    const float* W = wsh;
    float a = 0.f;
    if (t < F_H) {
      a = W[OFF_B1 + t];
      for (int i = 0; i < F_IN; ++i) a += x[i] * W[OFF_W1 + i * F_H + t];
      h1[t] = fmaxf(a, 0.f);
    }
    __syncthreads();
    if (t < F_H) {
      a = W[OFF_B2 + t];
      for (int i = 0; i < F_H; ++i) a += h1[i] * W[OFF_W2 + i * F_H + t];
      h2[t] = fmaxf(a, 0.f);
    }
    __syncthreads();
    if (t < F_OUT) {
      a = W[OFF_B3 + t];
      for (int i = 0; i < F_H; ++i) a += h2[i] * W[OFF_W3 + i * F_OUT + t];
      y[t] = a;
    }
    __syncthreads();
    if (t == 0) {
      int best = VAR_SLIMWORK;
      for (int v = 0; v < F_OUT; ++v) {
        if (v == VAR_PUSH && !push_fits(d, c)) continue;
        if (y[v] < y[best]) best = v;
      }
      // fallback: keep the frontier-size rule's choice unless the network
      // predicts a gain larger than the margin (in log-time units)
      int hv = choice;
      if (hv == VAR_PUSH && !push_fits(d, c)) hv = VAR_FILTERED;
      if (d.sel_margin > 0.0f && y[best] + d.sel_margin >= y[hv]) best = hv;
      choice = best;
    }
    __syncthreads();
  }
  if (t == 0) {
    int v = choice;
    if (v == VAR_PUSH && !push_fits(d, c)) v = VAR_FILTERED;
    // small frontiers go to the cluster push (several levels per launch)
    if (v == VAR_PUSH && local_fits(d, c->prev_new, c->prev_deg)) v = VAR_PUSH_LOCAL;
    c->variant = v;
    if (use_sw) cudaGraphSetConditional(sw, (unsigned)v);
  }
}

ss_status launch_decide(const slimsell_graph* h, const Dev& d, int policy,
                        cudaGraphConditionalHandle sw, int use_sw, cudaStream_t st) {
  k_decide<<<1, DECIDE_THREADS, 0, st>>>(d, policy, sw, use_sw, 0, 0);
  SS_CUDA(cudaGetLastError());
  return SS_OK;
}

ss_status add_decide_node(const slimsell_graph* h, const Dev& d, int policy,
                          cudaGraphConditionalHandle sw, cudaGraphConditionalHandle cw,
                          cudaGraph_t g, cudaGraphNode_t* out) {
  Dev dd = d;
  int pol = policy, use = 1, usew = 1;
  cudaGraphConditionalHandle hs = sw, hw = cw;
  void* args[] = {&dd, &pol, &hs, &use, &hw, &usew};
  cudaKernelNodeParams kp = {};
  kp.func = (void*)k_decide;
  kp.gridDim = dim3(1);
  kp.blockDim = dim3(DECIDE_THREADS);
  kp.sharedMemBytes = 0;
  kp.kernelParams = args;
  SS_CUDA(cudaGraphAddKernelNode(out, g, nullptr, 0, &kp));
  return SS_OK;
}

// ---------------------------------------------------------------------------
// MLP forward (batch) and one training step (forward, masked MSE, backward, Adam)
// ---------------------------------------------------------------------------
__global__ void k_mlp_forward(const float* __restrict__ W, const float* __restrict__ X, int B,
                              float* __restrict__ Y) {
  const int b = blockIdx.x * blockDim.x + threadIdx.x;
  if (b >= B) return;
  float x[F_IN], h1[F_H];
  for (int i = 0; i < F_IN; ++i) x[i] = X[(size_t)b * F_IN + i];
  for (int j = 0; j < F_H; ++j) {
    float a = W[OFF_B1 + j];
    for (int i = 0; i < F_IN; ++i) a += x[i] * W[OFF_W1 + i * F_H + j];
    h1[j] = fmaxf(a, 0.f);
  }
  float y[F_OUT];
  for (int o = 0; o < F_OUT; ++o) y[o] = W[OFF_B3 + o];
  for (int j = 0; j < F_H; ++j) {
    float a = W[OFF_B2 + j];
    for (int i = 0; i < F_H; ++i) a += h1[i] * W[OFF_W2 + i * F_H + j];
    a = fmaxf(a, 0.f);
    for (int o = 0; o < F_OUT; ++o) y[o] += a * W[OFF_W3 + j * F_OUT + o];
  }
  for (int o = 0; o < F_OUT; ++o) Y[(size_t)b * F_OUT + o] = y[o];
}

constexpr int TRAIN_THREADS = 256;
constexpr int TRAIN_MAX_BATCH = 128;

// Single block; B <= TRAIN_MAX_BATCH.  Loss = sum(mask * (y - t)^2) / max(sum(mask), 1).
__global__ void __launch_bounds__(TRAIN_THREADS) k_mlp_train(float* W, float* M, float* V, int step,
                                                              const float* X, const float* T,
                                                              const float* Mask, int B, float lr,
                                                              float* grad_out, float* loss_out) {
  extern __shared__ float sm[];
  float* x = sm;                       // [B][F_IN]
  float* h1 = x + B * F_IN;            // [B][F_H]
  float* h2 = h1 + B * F_H;            // [B][F_H]
  float* dy = h2 + B * F_H;            // [B][F_OUT]
  float* dh2 = dy + B * F_OUT;         // [B][F_H]
  float* dh1 = dh2 + B * F_H;          // [B][F_H]
  __shared__ float red[TRAIN_THREADS];
  const int t = threadIdx.x;
  for (int i = t; i < B * F_IN; i += TRAIN_THREADS) x[i] = X[i];
  __syncthreads();
  for (int e = t; e < B * F_H; e += TRAIN_THREADS) {
    const int b = e / F_H, j = e % F_H;
    float a = W[OFF_B1 + j];
    for (int i = 0; i < F_IN; ++i) a += x[b * F_IN + i] * W[OFF_W1 + i * F_H + j];
    h1[e] = fmaxf(a, 0.f);
  }
  __syncthreads();
  for (int e = t; e < B * F_H; e += TRAIN_THREADS) {
    const int b = e / F_H, j = e % F_H;
    float a = W[OFF_B2 + j];
    for (int i = 0; i < F_H; ++i) a += h1[b * F_H + i] * W[OFF_W2 + i * F_H + j];
    h2[e] = fmaxf(a, 0.f);
  }
  __syncthreads();
  // outputs, loss terms, dL/dy
  float msum = 0.f, lsum = 0.f;
  for (int e = 0; e < B * F_OUT; ++e) msum += Mask[e];  // every thread: same value
  const float denom = fmaxf(msum, 1.f);
  for (int e = t; e < B * F_OUT; e += TRAIN_THREADS) {
    const int b = e / F_OUT, o = e % F_OUT;
    float a = W[OFF_B3 + o];
    for (int j = 0; j < F_H; ++j) a += h2[b * F_H + j] * W[OFF_W3 + j * F_OUT + o];
    const float r = a - T[e];
    lsum += Mask[e] * r * r;
    dy[e] = 2.f * Mask[e] * r / denom;
  }
  red[t] = lsum;
  __syncthreads();
  for (int s = TRAIN_THREADS / 2; s > 0; s >>= 1) {
    if (t < s) red[t] += red[t + s];
    __syncthreads();
  }
  if (t == 0 && loss_out) *loss_out = red[0] / denom;
  // dh2 = dy W3^T * relu'(h2)
  for (int e = t; e < B * F_H; e += TRAIN_THREADS) {
    const int b = e / F_H, j = e % F_H;
    float a = 0.f;
    for (int o = 0; o < F_OUT; ++o) a += dy[b * F_OUT + o] * W[OFF_W3 + j * F_OUT + o];
    dh2[e] = h2[e] > 0.f ? a : 0.f;
  }
  __syncthreads();
  // dh1 = dh2 W2^T * relu'(h1)
  for (int e = t; e < B * F_H; e += TRAIN_THREADS) {
    const int b = e / F_H, i = e % F_H;
    float a = 0.f;
    for (int j = 0; j < F_H; ++j) a += dh2[b * F_H + j] * W[OFF_W2 + i * F_H + j];
    dh1[e] = h1[e] > 0.f ? a : 0.f;
  }
  __syncthreads();
  // parameter gradients (one thread per parameter), then Adam
  for (int p = t; p < N_PARAMS; p += TRAIN_THREADS) {
    float g = 0.f;
    if (p < OFF_B1) {
      const int i = p / F_H, j = p % F_H;
      for (int b = 0; b < B; ++b) g += x[b * F_IN + i] * dh1[b * F_H + j];
    } else if (p < OFF_W2) {
      const int j = p - OFF_B1;
      for (int b = 0; b < B; ++b) g += dh1[b * F_H + j];
    } else if (p < OFF_B2) {
      const int q = p - OFF_W2, i = q / F_H, j = q % F_H;
      for (int b = 0; b < B; ++b) g += h1[b * F_H + i] * dh2[b * F_H + j];
    } else if (p < OFF_W3) {
      const int j = p - OFF_B2;
      for (int b = 0; b < B; ++b) g += dh2[b * F_H + j];
    } else if (p < OFF_B3) {
      const int q = p - OFF_W3, j = q / F_OUT, o = q % F_OUT;
      for (int b = 0; b < B; ++b) g += h2[b * F_H + j] * dy[b * F_OUT + o];
    } else {
      const int o = p - OFF_B3;
      for (int b = 0; b < B; ++b) g += dy[b * F_OUT + o];
    }
    if (grad_out) grad_out[p] = g;
    if (lr > 0.f && M && V) {
      const float b1 = 0.9f, b2 = 0.999f, eps = 1e-8f;
      const float m = b1 * M[p] + (1.f - b1) * g;
      const float v = b2 * V[p] + (1.f - b2) * g * g;
      M[p] = m;
      V[p] = v;
      const float mh = m / (1.f - powf(b1, (float)step));
      const float vh = v / (1.f - powf(b2, (float)step));
      W[p] -= lr * mh / (sqrtf(vh) + eps);
    }
  }
}

}  // namespace ss

extern "C" {

ss_status slimsell_selector_load(slimsell_handle h, const float* h_weights, int64_t len) {
  if (!h) {
    ss::set_error("slimsell_selector_load: NULL handle");
    return SS_ERR_INVALID;
  }
  if (h->pending) SS_CUDA(cudaEventSynchronize(h->ev_done));  // a queued run may read the weights
  if (!h_weights) {  // unload: the learned policy falls back to the heuristic
    ss::drop_loop_graphs(h);  // captured loops hold the weight pointer
    if (h->mlp) cudaFree(h->mlp);
    h->mlp = nullptr;
    return SS_OK;
  }
  if (len != SS_SELECTOR_PARAMS) {
    ss::set_error("slimsell_selector_load: expected %d parameters, got %lld", SS_SELECTOR_PARAMS,
                  (long long)len);
    return SS_ERR_INVALID;
  }
  if (!h->mlp) {
    ss_status s = ss::dmalloc(h, (void**)&h->mlp, sizeof(float) * SS_SELECTOR_PARAMS);
    if (s != SS_OK) return s;
  }
  SS_CUDA(cudaMemcpy(h->mlp, h_weights, sizeof(float) * SS_SELECTOR_PARAMS, cudaMemcpyHostToDevice));
  ss::drop_loop_graphs(h);  // captured loops hold the old weight pointer
  return SS_OK;
}

ss_status slimsell_get_features(slimsell_handle h, float* h_out, int32_t cap) {
  if (!h || !h_out) {
    ss::set_error("slimsell_get_features: NULL argument");
    return SS_ERR_INVALID;
  }
  ss_run_stats st;
  ss_status s = slimsell_get_run_stats(h, &st, nullptr, 0);
  if (s != SS_OK) return s;
  int cnt = st.iterations + 1;
  if (cnt > cap) cnt = cap;
  if (cnt > h->iter_cap) cnt = h->iter_cap;
  SS_CUDA(cudaMemcpy(h_out, h->feats, sizeof(float) * SS_SELECTOR_FEATURES * (size_t)cnt,
                     cudaMemcpyDeviceToHost));
  return SS_OK;
}

ss_status slimsell_mlp_forward(const float* d_w, const float* d_x, int32_t batch, float* d_y,
                               void* stream) {
  if (!d_w || !d_x || !d_y || batch < 0) {
    ss::set_error("slimsell_mlp_forward: bad arguments");
    return SS_ERR_INVALID;
  }
  if (batch == 0) return SS_OK;
  ss::k_mlp_forward<<<(batch + 127) / 128, 128, 0, (cudaStream_t)stream>>>(d_w, d_x, batch, d_y);
  SS_CUDA(cudaGetLastError());
  return SS_OK;
}

ss_status slimsell_mlp_train_step(float* d_w, float* d_adam_m, float* d_adam_v, int32_t step,
                                  const float* d_x, const float* d_t, const float* d_mask,
                                  int32_t batch, float lr, float* d_grad, float* d_loss,
                                  void* stream) {
  using namespace ss;
  if (!d_w || !d_x || !d_t || !d_mask || batch < 1 || batch > TRAIN_MAX_BATCH || step < 1 ||
      (lr > 0.f && (!d_adam_m || !d_adam_v))) {
    set_error("slimsell_mlp_train_step: bad arguments (batch must be 1..%d, step >= 1)",
              TRAIN_MAX_BATCH);
    return SS_ERR_INVALID;
  }
  const size_t smem = sizeof(float) * (size_t)batch * (F_IN + 4 * F_H + F_OUT);
  static std::atomic<unsigned long long> configured{0};
  if (first_on_device(configured)) {
    const size_t maxsm = sizeof(float) * (size_t)TRAIN_MAX_BATCH * (F_IN + 4 * F_H + F_OUT);
    SS_CUDA(cudaFuncSetAttribute(k_mlp_train, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)maxsm));
  }
  k_mlp_train<<<1, TRAIN_THREADS, smem, (cudaStream_t)stream>>>(d_w, d_adam_m, d_adam_v, step, d_x,
                                                                 d_t, d_mask, batch, lr, d_grad,
                                                                 d_loss);
  SS_CUDA(cudaGetLastError());
  return SS_OK;
}

}  // extern "C"
