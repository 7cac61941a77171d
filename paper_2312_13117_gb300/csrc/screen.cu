// Learned screen: features from coarse indicators and a small MLP that decides
// which disks can skip the full indicator.
//
// Features of a disk (Eq. 3.1 at coarse resolutions): the ratio indicator with
// the first 8 and 16 nodes of an N-node rule (N a multiple of 16; the 8- and
// 16-node rules are sub-rules of every 16-divisible trapezoid rule on the same
// circle), plus the radius, all as log10. Label for training: the decision of
// the full rule, I_N > tol_ind.
//
// The network is 3 -> 64 -> 64 -> 1 with ReLU hidden layers and a sigmoid
// output. Master weights are FP32; the forward and backward passes read a BF16
// copy (round to nearest even) and accumulate in FP32. Training minimises a
// class-weighted binary cross-entropy with Adam. Each training step runs three
// deterministic kernels: per-sample forward and back-propagation to the hidden
// layers, parameter gradients as sums over the minibatch (one thread per
// parameter), and the Adam update with the BF16 refresh.
#include <cuda_bf16.h>

#include <cmath>
#include <cstring>
#include <vector>

#include "pmcim_internal.cuh"

namespace {

constexpr int H = 64;
// parameter layout (floats): W1[H][3] b1[H] W2[H][H] b2[H] W3[H] b3
constexpr int O_W1 = 0, O_B1 = O_W1 + H * 3, O_W2 = O_B1 + H, O_B2 = O_W2 + H * H, O_W3 = O_B2 + H,
              O_B3 = O_W3 + H, NPARAM = O_B3 + 1;
static_assert(NPARAM == PMCIM_SCREEN_PARAMS, "parameter count");

// ---------------------------------------------------------------------------
// Multi-resolution indicator: I_8, I_16, I_N of every disk from its node
// solutions (column 0 of X, i.e. f = V[:,0]).
// ---------------------------------------------------------------------------
constexpr int FT = 256;

// P f|_M and P f|_{M/2} (component i) on the M-node rule of disk rg, whose node m is
// node m * (N / M) of the disk's N-node rule; s_abs = sum_m |w_m| |x_m|.
__device__ __forceinline__ void pf_component(const LevelArgs& a, const RegionDev& rg, size_t nl, int M, int i,
                                             double2* s_full, double2* s_half, double* s_abs) {
  const int step = rg.N / M;
  double2 f = make_double2(0.0, 0.0), h = f;
  double ab = 0.0;
  for (int m = 0; m < M; ++m) {
    double2 z, w;
    node_weight(rg.cre, rg.cim, rg.r, M, m, &z, &w);
    const double2 x = a.X[rg.x_off + (size_t)(m * step) * nl + i];
    cfma(f, w, x);
    if (m & 1) cfma(h, cscale(w, 2.0), x);
    ab += hypot(w.x, w.y) * hypot(x.x, x.y);
  }
  *s_full = f;
  *s_half = h;
  *s_abs = ab;
}

// The indicator of Eq. 3.1 at three resolutions, with the reading the indicator
// kernel takes: 0 when P f|_M is at rounding level as a whole, else the root mean
// square of the componentwise ratios whose P f|_{M/2} is above that level.
__global__ void __launch_bounds__(FT) k_screen_features(LevelArgs a, double* ind3) {
  __shared__ double red[6][FT / 32];
  __shared__ double tot[6];
  const int g = blockIdx.x;
  const RegionDev rg = a.regions[g];
  const ProblemDev* P = a.probs + rg.prob;
  const int n = P->n, l = P->l, N = rg.N;
  const size_t nl = (size_t)n * l;
  const int res[3] = {8, 16, N};
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  // pass 1, per resolution: ||P f_M||^2 and ||sum |w||x| ||^2
  double acc[6] = {0.0, 0.0, 0.0, 0.0, 0.0, 0.0};
  for (int i = threadIdx.x; i < n; i += FT)
    for (int q = 0; q < 3; ++q) {
      double2 f, h;
      double ab;
      pf_component(a, rg, nl, res[q], i, &f, &h, &ab);
      acc[2 * q] += cabs2(f);
      acc[2 * q + 1] += ab * ab;
    }
  for (int q = 0; q < 6; ++q)
    for (int o = 16; o > 0; o >>= 1) acc[q] += __shfl_down_sync(0xffffffffu, acc[q], o);
  if (lane == 0)
    for (int q = 0; q < 6; ++q) red[q][wid] = acc[q];
  __syncthreads();
  if (threadIdx.x < 6) {
    double t = 0.0;
    for (int k = 0; k < FT / 32; ++k) t += red[threadIdx.x][k];
    tot[threadIdx.x] = t;
  }
  __syncthreads();
  // pass 2, per resolution: sum of the determined |ratio|^2 and their count
  double acc2[6] = {0.0, 0.0, 0.0, 0.0, 0.0, 0.0};
  for (int i = threadIdx.x; i < n; i += FT)
    for (int q = 0; q < 3; ++q) {
      double2 f, h;
      double ab;
      pf_component(a, rg, nl, res[q], i, &f, &h, &ab);
      const double den = cabs2(h);
      if (den > kPfFloor * kPfFloor * tot[2 * q + 1]) {
        acc2[2 * q] += cabs2(f) / den;
        acc2[2 * q + 1] += 1.0;
      }
    }
  for (int q = 0; q < 6; ++q)
    for (int o = 16; o > 0; o >>= 1) acc2[q] += __shfl_down_sync(0xffffffffu, acc2[q], o);
  __syncthreads();
  if (lane == 0)
    for (int q = 0; q < 6; ++q) red[q][wid] = acc2[q];
  __syncthreads();
  if (threadIdx.x < 3) {
    const int q = threadIdx.x;
    double sr = 0.0, kept = 0.0;
    for (int k = 0; k < FT / 32; ++k) {
      sr += red[2 * q][k];
      kept += red[2 * q + 1][k];
    }
    // P f at rounding level: indicator 0 (Sec. 2.1: P f = 0 without eigenvalues)
    ind3[(size_t)g * 3 + q] =
        (sqrt(tot[2 * q]) <= kPfFloor * sqrt(tot[2 * q + 1]) || kept == 0.0) ? 0.0 : sqrt(sr / kept);
  }
}

// ---------------------------------------------------------------------------
// MLP kernels
// ---------------------------------------------------------------------------
constexpr int MT = 128;

__device__ __forceinline__ float relu(float x) { return x > 0.f ? x : 0.f; }

// BF16 weights -> FP32 in shared memory
__device__ void load_weights(float* sw, const __nv_bfloat16* wb) {
  for (int i = threadIdx.x; i < NPARAM; i += blockDim.x) sw[i] = __bfloat162float(wb[i]);
  __syncthreads();
}

// logit of one sample (h1 kept in registers, h2 produced one unit at a time)
__device__ float forward_logit(const float* sw, const float x[3], float h1[H]) {
#pragma unroll
  for (int j = 0; j < H; ++j) {
    float v = sw[O_B1 + j];
#pragma unroll
    for (int i = 0; i < 3; ++i) v = fmaf(sw[O_W1 + j * 3 + i], x[i], v);
    h1[j] = relu(v);
  }
  float o = sw[O_B3];
  for (int k = 0; k < H; ++k) {
    float v = sw[O_B2 + k];
#pragma unroll
    for (int j = 0; j < H; ++j) v = fmaf(sw[O_W2 + k * H + j], h1[j], v);
    o = fmaf(sw[O_W3 + k], relu(v), o);
  }
  return o;
}

__global__ void __launch_bounds__(MT) k_mlp_forward(int M, const float* __restrict__ feats,
                                                     const __nv_bfloat16* __restrict__ wb, float* __restrict__ prob) {
  __shared__ float sw[NPARAM];
  load_weights(sw, wb);
  const int b = blockIdx.x * MT + threadIdx.x;
  if (b >= M) return;
  const float x[3] = {feats[3 * b], feats[3 * b + 1], feats[3 * b + 2]};
  float h1[H];
  const float o = forward_logit(sw, x, h1);
  prob[b] = 1.f / (1.f + expf(-o));
}

// Per sample: forward, loss, and the back-propagated signals of the two hidden
// layers (dh2 = dL/d(pre-activation of layer 2), dh1 likewise), stored for the
// parameter-gradient kernel together with h1 and h2.
__global__ void __launch_bounds__(MT) k_mlp_fwd_bwd(int B, const float* __restrict__ feats,
                                                     const uint8_t* __restrict__ labels, float pos_weight,
                                                     const __nv_bfloat16* __restrict__ wb, float* __restrict__ H1,
                                                     float* __restrict__ H2, float* __restrict__ D2,
                                                     float* __restrict__ D1, float* __restrict__ DO,
                                                     float* __restrict__ loss) {
  __shared__ float sw[NPARAM];
  load_weights(sw, wb);
  const int b = blockIdx.x * MT + threadIdx.x;
  if (b >= B) return;
  const float x[3] = {feats[3 * b], feats[3 * b + 1], feats[3 * b + 2]};
  float h1[H], h2[H];
#pragma unroll
  for (int j = 0; j < H; ++j) {
    float v = sw[O_B1 + j];
#pragma unroll
    for (int i = 0; i < 3; ++i) v = fmaf(sw[O_W1 + j * 3 + i], x[i], v);
    h1[j] = relu(v);
  }
  float o = sw[O_B3];
  for (int k = 0; k < H; ++k) {
    float v = sw[O_B2 + k];
#pragma unroll
    for (int j = 0; j < H; ++j) v = fmaf(sw[O_W2 + k * H + j], h1[j], v);
    h2[k] = relu(v);
    o = fmaf(sw[O_W3 + k], h2[k], o);
  }
  // weighted binary cross-entropy on the logit, in a stable form
  const float y = labels[b] ? 1.f : 0.f;
  const float wgt = labels[b] ? pos_weight : 1.f;
  const float sp = fmaxf(o, 0.f) + log1pf(expf(-fabsf(o)));  // log(1 + e^o)
  loss[b] = wgt * (sp - y * o);
  const float p = 1.f / (1.f + expf(-o));
  const float d_o = wgt * (p - y);
  DO[b] = d_o;
  float d1[H];
#pragma unroll
  for (int j = 0; j < H; ++j) d1[j] = 0.f;
  for (int k = 0; k < H; ++k) {
    const float d2 = h2[k] > 0.f ? d_o * sw[O_W3 + k] : 0.f;
    D2[(size_t)b * H + k] = d2;
    H2[(size_t)b * H + k] = h2[k];
#pragma unroll
    for (int j = 0; j < H; ++j) d1[j] = fmaf(d2, sw[O_W2 + k * H + j], d1[j]);
  }
#pragma unroll
  for (int j = 0; j < H; ++j) {
    D1[(size_t)b * H + j] = h1[j] > 0.f ? d1[j] : 0.f;
    H1[(size_t)b * H + j] = h1[j];
  }
}

// One thread per parameter: gradient = sum over the minibatch (fixed order);
// the minibatch mean is taken by dividing by B.
__global__ void k_mlp_param_grad(int B, const float* __restrict__ feats, const float* __restrict__ H1,
                                 const float* __restrict__ H2, const float* __restrict__ D2,
                                 const float* __restrict__ D1, const float* __restrict__ DO,
                                 float* __restrict__ grad) {
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= NPARAM) return;
  float s = 0.f;
  if (t < O_B1) {
    const int j = t / 3, i = t % 3;
    for (int b = 0; b < B; ++b) s = fmaf(D1[(size_t)b * H + j], feats[3 * b + i], s);
  } else if (t < O_W2) {
    const int j = t - O_B1;
    for (int b = 0; b < B; ++b) s += D1[(size_t)b * H + j];
  } else if (t < O_B2) {
    const int k = (t - O_W2) / H, j = (t - O_W2) % H;
    for (int b = 0; b < B; ++b) s = fmaf(D2[(size_t)b * H + k], H1[(size_t)b * H + j], s);
  } else if (t < O_W3) {
    const int k = t - O_B2;
    for (int b = 0; b < B; ++b) s += D2[(size_t)b * H + k];
  } else if (t < O_B3) {
    const int k = t - O_W3;
    for (int b = 0; b < B; ++b) s = fmaf(DO[b], H2[(size_t)b * H + k], s);
  } else {
    for (int b = 0; b < B; ++b) s += DO[b];
  }
  grad[t] = s / (float)B;
}

__global__ void k_sum(int B, const float* __restrict__ v, double* __restrict__ out) {
  __shared__ double red[256];
  double s = 0.0;
  for (int i = threadIdx.x; i < B; i += 256) s += v[i];
  red[threadIdx.x] = s;
  __syncthreads();
  for (int w = 128; w > 0; w >>= 1) {
    if (threadIdx.x < w) red[threadIdx.x] += red[threadIdx.x + w];
    __syncthreads();
  }
  if (threadIdx.x == 0) *out = red[0] / (double)B;
}

// Adam (Kingma & Ba) on the FP32 master weights, then the BF16 copy.
__global__ void k_adam(float* __restrict__ w, float* __restrict__ m, float* __restrict__ v,
                       const float* __restrict__ g, __nv_bfloat16* __restrict__ wb, float lr, float b1, float b2,
                       float eps, float c1, float c2) {
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= NPARAM) return;
  const float gt = g[t];
  const float mt = b1 * m[t] + (1.f - b1) * gt;
  const float vt = b2 * v[t] + (1.f - b2) * gt * gt;
  m[t] = mt;
  v[t] = vt;
  const float wt = w[t] - lr * (mt / c1) / (sqrtf(vt / c2) + eps);
  w[t] = wt;
  wb[t] = __float2bfloat16_rn(wt);
}

__global__ void k_to_bf16(int n, const float* __restrict__ w, __nv_bfloat16* __restrict__ wb) {
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t < n) wb[t] = __float2bfloat16_rn(w[t]);
}

// Features (log10 I_8, log10 I_16, log10 r) of every disk from the indicators.
__global__ void k_make_features(int R, const double* __restrict__ ind3, const RegionDev* __restrict__ regions,
                                float* __restrict__ feats) {
  const int g = blockIdx.x * blockDim.x + threadIdx.x;
  if (g >= R) return;
  feats[3 * g] = (float)log10(fmax(ind3[3 * g], 1e-30));
  feats[3 * g + 1] = (float)log10(fmax(ind3[3 * g + 1], 1e-30));
  feats[3 * g + 2] = (float)log10(regions[g].r);
}

}  // namespace

cudaError_t launch_screen_features(const LevelArgs& a, double* ind3, cudaStream_t s) {
  if (a.R <= 0) return cudaSuccess;
  k_screen_features<<<a.R, FT, 0, s>>>(a, ind3);
  return cudaGetLastError();
}

cudaError_t launch_make_features(int R, const double* ind3, const RegionDev* regions, float* feats, cudaStream_t s) {
  if (R <= 0) return cudaSuccess;
  k_make_features<<<(R + 255) / 256, 256, 0, s>>>(R, ind3, regions, feats);
  return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// Host side of the MLP (device buffers only; the C ABI wraps these in api.cu)
// ---------------------------------------------------------------------------
cudaError_t screen_forward(int M, const float* d_feats, const float* d_params, float* d_prob, void* d_scratch,
                           cudaStream_t s) {
  if (M <= 0) return cudaSuccess;
  __nv_bfloat16* wb = reinterpret_cast<__nv_bfloat16*>(d_scratch);
  k_to_bf16<<<(NPARAM + 255) / 256, 256, 0, s>>>(NPARAM, d_params, wb);
  k_mlp_forward<<<(M + MT - 1) / MT, MT, 0, s>>>(M, d_feats, wb, d_prob);
  return cudaGetLastError();
}

// Scratch of one gradient evaluation: BF16 weights, then per-sample H1, H2, D2,
// D1 (B x 64 each), the output signal and the loss (B each).
size_t screen_grad_scratch_bytes(int B) {
  return (((size_t)NPARAM * 2 + 255) & ~(size_t)255) + (size_t)B * (4 * H + 2) * sizeof(float);
}

// Scratch of training: gradient, Adam moments (NPARAM floats each), two
// doubles, then one gradient evaluation's scratch.
size_t screen_train_scratch_bytes(int B) {
  return (((size_t)NPARAM * 3 * 4 + 64 + 255) & ~(size_t)255) + screen_grad_scratch_bytes(B);
}

// Gradient of the mean weighted loss at the BF16 rounding of params (one minibatch).
cudaError_t screen_gradient(int B, const float* d_feats, const uint8_t* d_labels, float pos_weight,
                            const float* d_params, float* d_grad, double* d_loss, void* d_scratch, cudaStream_t s) {
  char* p = reinterpret_cast<char*>(d_scratch);
  __nv_bfloat16* wb = reinterpret_cast<__nv_bfloat16*>(p);
  p += ((size_t)NPARAM * 2 + 255) & ~(size_t)255;
  float* H1 = reinterpret_cast<float*>(p);
  float* H2 = H1 + (size_t)B * H;
  float* D2 = H2 + (size_t)B * H;
  float* D1 = D2 + (size_t)B * H;
  float* DO = D1 + (size_t)B * H;
  float* LS = DO + B;
  k_to_bf16<<<(NPARAM + 255) / 256, 256, 0, s>>>(NPARAM, d_params, wb);
  k_mlp_fwd_bwd<<<(B + MT - 1) / MT, MT, 0, s>>>(B, d_feats, d_labels, pos_weight, wb, H1, H2, D2, D1, DO, LS);
  k_mlp_param_grad<<<(NPARAM + 127) / 128, 128, 0, s>>>(B, d_feats, H1, H2, D2, D1, DO, d_grad);
  if (d_loss) k_sum<<<1, 256, 0, s>>>(B, LS, d_loss);
  return cudaGetLastError();
}

__global__ void k_accumulate(double* dst, const double* src, double w) { *dst += w * *src; }

// Adam over `epochs` passes of the data in minibatches of B (in the given
// order). d_epoch_loss[ep] receives the epoch's mean weighted loss.
cudaError_t screen_train(int M, const float* d_feats, const uint8_t* d_labels, int epochs, int B, float lr,
                         float pos_weight, float* d_params, double* d_epoch_loss, void* d_scratch, cudaStream_t s) {
  char* base = reinterpret_cast<char*>(d_scratch);
  float* grad = reinterpret_cast<float*>(base);
  float* mom = grad + NPARAM;
  float* var = mom + NPARAM;
  double* bl = reinterpret_cast<double*>(base + (size_t)NPARAM * 3 * 4 + 8 - ((size_t)NPARAM * 3 * 4) % 8);
  void* inner = base + (((size_t)NPARAM * 3 * 4 + 64 + 255) & ~(size_t)255);
  __nv_bfloat16* wb = reinterpret_cast<__nv_bfloat16*>(inner);
  cudaError_t e = cudaMemsetAsync(mom, 0, 2 * (size_t)NPARAM * sizeof(float), s);
  if (e != cudaSuccess) return e;
  const float b1 = 0.9f, b2 = 0.999f, eps = 1e-8f;
  int t = 0;
  for (int ep = 0; ep < epochs; ++ep) {
    if (d_epoch_loss) {
      e = cudaMemsetAsync(d_epoch_loss + ep, 0, sizeof(double), s);
      if (e != cudaSuccess) return e;
    }
    for (int b0 = 0; b0 < M; b0 += B) {
      const int bs = (M - b0) < B ? (M - b0) : B;
      e = screen_gradient(bs, d_feats + 3 * (size_t)b0, d_labels + b0, pos_weight, d_params, grad,
                          d_epoch_loss ? bl : nullptr, inner, s);
      if (e != cudaSuccess) return e;
      ++t;
      const float c1 = 1.f - powf(b1, (float)t), c2 = 1.f - powf(b2, (float)t);
      k_adam<<<(NPARAM + 255) / 256, 256, 0, s>>>(d_params, mom, var, grad, wb, lr, b1, b2, eps, c1, c2);
      if (d_epoch_loss) k_accumulate<<<1, 1, 0, s>>>(d_epoch_loss + ep, bl, (double)bs / (double)M);
    }
  }
  return cudaGetLastError();
}
