// Learned preconditioner network: conv3d(2->16) ReLU conv3d(16->16) ReLU conv3d(16->1),
// 3^3 kernels, stride 1, zero padding 1; weights rounded to bf16 for every use (FP32
// masters updated by Adam), FP32 activations and accumulation.  The paper has no
// learned component; this is the eigensolver preconditioner the project adds.
//
// Kernels: k_conv_fwd (direct convolution, a CTA computes an 8 x 8 x 8 output block for
// all output channels from a shared-memory halo tile), the data gradient as the same
// convolution with flipped, transposed weights (k_flip_weights), k_conv_wgrad (per-block
// partial sums, reduced in fixed order by k_wgrad_reduce), masked MSE loss, ReLU
// backward and Adam.
#include <cuda_runtime.h>

#include <cmath>
#include <cstdint>
#include <cstdio>
#include <cstring>
#include <vector>

#include "../../include/rsx.h"
#include "api_internal.cuh"

namespace {

constexpr int kC1 = 2, kC2 = 16, kC3 = 16, kC4 = 1;   // channels in -> hidden -> hidden -> out
constexpr int kT = 8;                                   // output block edge
constexpr int kHalo = kT + 2;
constexpr int kConvThreads = 256;
// parameter layout (floats): w1 [16][2][27], b1 [16], w2 [16][16][27], b2 [16], w3 [1][16][27], b3 [1]
constexpr int kW1 = kC2 * kC1 * 27, kW2 = kC3 * kC2 * 27, kW3 = kC4 * kC3 * 27;
constexpr int kOffW1 = 0, kOffB1 = kW1, kOffW2 = kOffB1 + kC2, kOffB2 = kOffW2 + kW2, kOffW3 = kOffB2 + kC3,
              kOffB3 = kOffW3 + kW3, kNParams = kOffB3 + kC4;

__device__ __forceinline__ float bf16_round(float f) {
  const uint32_t u = __float_as_uint(f);
  return __uint_as_float(((u + 0x7FFFu + ((u >> 16) & 1u)) >> 16) << 16);
}

// out[b][co][v] = bias[co] + sum_{ci,tap} w[co][ci][tap] * act(in[b][ci][v + tap - 1])
// act = ReLU on the input when relu_in (the previous layer's activation).
// Grid: (blocks of 8^3) x B.  Each thread owns 2 voxels (z, z+4) x CO outputs.
template <int CI, int CO>
__global__ void __launch_bounds__(kConvThreads) k_conv_fwd(const float* __restrict__ in, const float* __restrict__ w,
                                                           const float* __restrict__ bias, float* __restrict__ out,
                                                           int D, int H, int W, int relu_in) {
  constexpr int CCH = CI < 4 ? CI : 4;   // input channels staged per round
  __shared__ float tile[CCH][kHalo][kHalo][kHalo];
  __shared__ float ws[CO][CCH][27];
  const int nbx = (W + kT - 1) / kT, nby = (H + kT - 1) / kT;
  int blk = blockIdx.x;
  const int bx = blk % nbx;
  blk /= nbx;
  const int by = blk % nby;
  const int bz = blk / nby;
  const int b = blockIdx.y;
  const int x0 = bx * kT, y0 = by * kT, z0 = bz * kT;
  const int tx = threadIdx.x & 7, ty = (threadIdx.x >> 3) & 7, tz = threadIdx.x >> 6;  // tz 0..3
  const size_t vol = (size_t)D * H * W;
  float acc0[CO], acc1[CO];
#pragma unroll
  for (int o = 0; o < CO; ++o) acc0[o] = acc1[o] = bias ? bias[o] : 0.f;
  for (int c0 = 0; c0 < CI; c0 += CCH) {
    __syncthreads();
    for (int i = threadIdx.x; i < CCH * kHalo * kHalo * kHalo; i += kConvThreads) {
      const int c = i / (kHalo * kHalo * kHalo);
      int r = i - c * kHalo * kHalo * kHalo;
      const int hz = r / (kHalo * kHalo);
      r -= hz * kHalo * kHalo;
      const int hy = r / kHalo, hx = r - hy * kHalo;
      const int z = z0 + hz - 1, y = y0 + hy - 1, x = x0 + hx - 1;
      float v = 0.f;
      if (c0 + c < CI && z >= 0 && z < D && y >= 0 && y < H && x >= 0 && x < W) {
        v = in[((size_t)b * CI + c0 + c) * vol + ((size_t)z * H + y) * W + x];
        if (relu_in) v = fmaxf(v, 0.f);
      }
      tile[c][hz][hy][hx] = v;
    }
    for (int i = threadIdx.x; i < CO * CCH * 27; i += kConvThreads) {
      const int o = i / (CCH * 27), r = i - o * CCH * 27, c = r / 27, t = r - c * 27;
      ws[o][c][t] = (c0 + c < CI) ? bf16_round(w[((size_t)o * CI + c0 + c) * 27 + t]) : 0.f;
    }
    __syncthreads();
#pragma unroll 1
    for (int c = 0; c < CCH; ++c) {
#pragma unroll
      for (int t = 0; t < 27; ++t) {
        const int dz = t / 9, dy = (t / 3) % 3, dx = t % 3;
        const float a0 = tile[c][tz + dz][ty + dy][tx + dx];
        const float a1 = tile[c][tz + 4 + dz][ty + dy][tx + dx];
#pragma unroll
        for (int o = 0; o < CO; ++o) {
          const float wv = ws[o][c][t];
          acc0[o] = fmaf(wv, a0, acc0[o]);
          acc1[o] = fmaf(wv, a1, acc1[o]);
        }
      }
    }
  }
  const int x = x0 + tx, y = y0 + ty, za = z0 + tz, zb = z0 + tz + 4;
  if (x < W && y < H) {
#pragma unroll
    for (int o = 0; o < CO; ++o) {
      float* ob = out + ((size_t)b * CO + o) * vol;
      if (za < D) ob[((size_t)za * H + y) * W + x] = acc0[o];
      if (zb < D) ob[((size_t)zb * H + y) * W + x] = acc1[o];
    }
  }
}

// wt[ci][co][26 - t] = w[co][ci][t]: the data gradient is the forward convolution of
// dout with these weights (no bias)
__global__ void k_flip_weights(const float* __restrict__ w, float* __restrict__ wt, int CI, int CO) {
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < CI * CO * 27; i += gridDim.x * blockDim.x) {
    const int co = i / (CI * 27), r = i - co * CI * 27, ci = r / 27, t = r - ci * 27;
    wt[((size_t)ci * CO + co) * 27 + (26 - t)] = w[i];
  }
}

// dz = da * (z > 0)  (ReLU backward), in place on da
__global__ void k_relu_back(float* __restrict__ da, const float* __restrict__ z, size_t n) {
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x)
    if (!(z[i] > 0.f)) da[i] = 0.f;
}

// partial weight and bias gradients of one layer over one 8^3 block of one sample:
// part[blk][co][ci][t] = sum_v dout[co][v] act(in[ci][v + t - 1]), part[blk][CO*CI*27 + co] = sum_v dout[co][v]
template <int CI, int CO>
__global__ void __launch_bounds__(kConvThreads) k_conv_wgrad(const float* __restrict__ in, const float* __restrict__ dout,
                                                             float* __restrict__ part, int D, int H, int W, int relu_in) {
  __shared__ float tile[kHalo][kHalo][kHalo];
  __shared__ float dsh[CO][kT * kT * kT];
  const int nbx = (W + kT - 1) / kT, nby = (H + kT - 1) / kT, nbz = (D + kT - 1) / kT;
  int blk = blockIdx.x;
  const int bx = blk % nbx;
  blk /= nbx;
  const int by = blk % nby;
  const int bz = blk / nby;
  const int b = blockIdx.y;
  const int x0 = bx * kT, y0 = by * kT, z0 = bz * kT;
  const size_t vol = (size_t)D * H * W;
  constexpr int NOUT = CO * CI * 27 + CO;
  float* dst = part + ((size_t)b * nbx * nby * nbz + blockIdx.x) * NOUT;
  // stage dout block (zero outside)
  for (int i = threadIdx.x; i < CO * kT * kT * kT; i += kConvThreads) {
    const int o = i / (kT * kT * kT), v = i - o * kT * kT * kT;
    const int tz = v / (kT * kT), ty = (v / kT) % kT, tx = v % kT;
    const int z = z0 + tz, y = y0 + ty, x = x0 + tx;
    dsh[o][v] = (z < D && y < H && x < W) ? dout[((size_t)b * CO + o) * vol + ((size_t)z * H + y) * W + x] : 0.f;
  }
  for (int ci = 0; ci < CI; ++ci) {
    __syncthreads();
    for (int i = threadIdx.x; i < kHalo * kHalo * kHalo; i += kConvThreads) {
      const int hz = i / (kHalo * kHalo), hy = (i / kHalo) % kHalo, hx = i % kHalo;
      const int z = z0 + hz - 1, y = y0 + hy - 1, x = x0 + hx - 1;
      float v = 0.f;
      if (z >= 0 && z < D && y >= 0 && y < H && x >= 0 && x < W) {
        v = in[((size_t)b * CI + ci) * vol + ((size_t)z * H + y) * W + x];
        if (relu_in) v = fmaxf(v, 0.f);
      }
      tile[hz][hy][hx] = v;
    }
    __syncthreads();
    // outputs (co, t) for this ci: CO * 27 <= 432 -> threads loop
    for (int o = threadIdx.x; o < CO * 27; o += kConvThreads) {
      const int co = o / 27, t = o - co * 27;
      const int dz = t / 9, dy = (t / 3) % 3, dx = t % 3;
      float s = 0.f;
      for (int v = 0; v < kT * kT * kT; ++v) {
        const int tz = v / (kT * kT), ty = (v / kT) % kT, tx = v % kT;
        s = fmaf(dsh[co][v], tile[tz + dz][ty + dy][tx + dx], s);
      }
      dst[((size_t)co * CI + ci) * 27 + t] = s;
    }
  }
  __syncthreads();
  for (int co = threadIdx.x; co < CO; co += kConvThreads) {
    float s = 0.f;
    for (int v = 0; v < kT * kT * kT; ++v) s += dsh[co][v];
    dst[CO * CI * 27 + co] = s;
  }
}

// grad[o] (+)= sum over nparts of part[p][o], FP64 accumulation in fixed order
__global__ void k_wgrad_reduce(const float* __restrict__ part, int nparts, int nout, float* __restrict__ gw,
                               float* __restrict__ gb, int nw) {
  for (int o = blockIdx.x * blockDim.x + threadIdx.x; o < nout; o += gridDim.x * blockDim.x) {
    double s = 0.0;
    for (int p = 0; p < nparts; ++p) s += part[(size_t)p * nout + o];
    if (o < nw)
      gw[o] = (float)s;
    else
      gb[o - nw] = (float)s;
  }
}

// masked mean squared error: loss = sum m (y - t)^2 / sum m over the batch; dy = 2 m (y - t) / sum m.
// The mask excludes `border` voxels at every face of each sample.
__global__ void k_mse(const float* __restrict__ y, const float* __restrict__ t, float* __restrict__ dy, int B, int D,
                      int H, int W, int border, double* __restrict__ loss_acc) {
  const size_t vol = (size_t)D * H * W;
  const double cnt = (double)B * (D - 2 * border) * (H - 2 * border) * (W - 2 * border);
  double s = 0.0;
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < (size_t)B * vol;
       i += (size_t)gridDim.x * blockDim.x) {
    const size_t v = i % vol;
    const int x = (int)(v % W), yy = (int)((v / W) % H), z = (int)(v / ((size_t)W * H));
    const bool in = x >= border && x < W - border && yy >= border && yy < H - border && z >= border && z < D - border;
    const float d = in ? y[i] - t[i] : 0.f;
    dy[i] = (float)(2.0 * d / cnt);
    s += (double)d * d;
  }
  for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
  if ((threadIdx.x & 31) == 0) atomicAdd(loss_acc, s / cnt);
}

__global__ void k_adam(float* __restrict__ p, const float* __restrict__ g, float* __restrict__ m, float* __restrict__ v,
                       int n, float lr, float b1, float b2, float eps, float c1, float c2) {
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
    const float gi = g[i];
    const float mi = b1 * m[i] + (1.f - b1) * gi;
    const float vi = b2 * v[i] + (1.f - b2) * gi * gi;
    m[i] = mi;
    v[i] = vi;
    p[i] -= lr * (mi / c1) / (sqrtf(vi / c2) + eps);
  }
}

}  // namespace

struct rsx_net {
  int device = 0;
  float* params = nullptr;   // FP32 masters
  float* grads = nullptr;
  float* adam_m = nullptr;
  float* adam_v = nullptr;
  float* wflip = nullptr;    // flipped weights of one layer (scratch)
  float* act = nullptr;      // z1, z2 [B][16][vol] each
  size_t act_elems = 0;
  float* gout = nullptr;     // gradients of activations [B][16][vol] x 2 + output
  size_t gout_elems = 0;
  float* part = nullptr;
  size_t part_elems = 0;
  double* loss = nullptr;
  long long step = 0;
  char err[256] = {0};
};

namespace {

int nfail(rsx_net* n, int code, const char* msg) {
  snprintf(n->err, sizeof(n->err), "%s", msg);
  return code;
}

int ncuda(rsx_net* n, cudaError_t e, const char* what) {
  if (e == cudaSuccess) return RSX_OK;
  snprintf(n->err, sizeof(n->err), "%s: %s", what, cudaGetErrorString(e));
  return RSX_ECUDA;
}

int ngrow(rsx_net* n, float** p, size_t* have, size_t need) {
  if (need <= *have) return RSX_OK;
  if (*p) cudaFree(*p);
  *p = nullptr;
  *have = 0;
  if (cudaMalloc(p, need * sizeof(float)) != cudaSuccess) {
    cudaGetLastError();
    return nfail(n, RSX_ENOMEM, "network workspace allocation failed");
  }
  *have = need;
  return RSX_OK;
}

dim3 conv_grid(int B, int D, int H, int W) {
  return dim3((unsigned)(((W + kT - 1) / kT) * ((H + kT - 1) / kT) * ((D + kT - 1) / kT)), (unsigned)B);
}

int forward(rsx_net* n, const float* x, int B, int D, int H, int W, float* out, cudaStream_t s) {
  const size_t vol = (size_t)D * H * W;
  int rc = ngrow(n, &n->act, &n->act_elems, 2 * (size_t)B * kC2 * vol);
  if (rc) return rc;
  float* z1 = n->act;
  float* z2 = n->act + (size_t)B * kC2 * vol;
  const dim3 g = conv_grid(B, D, H, W);
  const float* P = n->params;
  k_conv_fwd<kC1, kC2><<<g, kConvThreads, 0, s>>>(x, P + kOffW1, P + kOffB1, z1, D, H, W, 0);
  k_conv_fwd<kC2, kC3><<<g, kConvThreads, 0, s>>>(z1, P + kOffW2, P + kOffB2, z2, D, H, W, 1);
  k_conv_fwd<kC3, kC4><<<g, kConvThreads, 0, s>>>(z2, P + kOffW3, P + kOffB3, out, D, H, W, 1);
  return ncuda(n, cudaGetLastError(), "network forward");
}

// gradients of the masked MSE loss w.r.t. all parameters into n->grads; loss (device double) += value
int backward(rsx_net* n, const float* x, const float* target, int B, int D, int H, int W, int border, cudaStream_t s) {
  const size_t vol = (size_t)D * H * W;
  int rc = ngrow(n, &n->gout, &n->gout_elems, 2 * (size_t)B * kC2 * vol + (size_t)B * vol * 2);
  if (rc) return rc;
  const int nblk = ((W + kT - 1) / kT) * ((H + kT - 1) / kT) * ((D + kT - 1) / kT);
  rc = ngrow(n, &n->part, &n->part_elems, (size_t)B * nblk * (kW2 + kC3));
  if (rc) return rc;
  float* g2 = n->gout;                                  // d z2  [B][16][vol]
  float* g1 = n->gout + (size_t)B * kC2 * vol;          // d z1  [B][16][vol]
  float* y = g1 + (size_t)B * kC2 * vol;                // output [B][vol]
  float* gy = y + (size_t)B * vol;                      // d output
  rc = forward(n, x, B, D, H, W, y, s);                 // (re)sizes n->act
  if (rc) return rc;
  float* z1 = n->act;                                   // pre-activations of layers 1 and 2
  float* z2 = n->act + (size_t)B * kC2 * vol;
  k_mse<<<512, 256, 0, s>>>(y, target, gy, B, D, H, W, border, n->loss);
  const dim3 g = conv_grid(B, D, H, W);
  const float* P = n->params;
  // layer 3: w3 grads from relu(z2) and gy; d relu(z2) = conv(gy, flip(w3)); dz2 = * (z2 > 0)
  k_conv_wgrad<kC3, kC4><<<g, kConvThreads, 0, s>>>(z2, gy, n->part, D, H, W, 1);
  k_wgrad_reduce<<<64, 256, 0, s>>>(n->part, B * nblk, kW3 + kC4, n->grads + kOffW3, n->grads + kOffB3, kW3);
  k_flip_weights<<<16, 256, 0, s>>>(P + kOffW3, n->wflip, kC3, kC4);
  k_conv_fwd<kC4, kC3><<<g, kConvThreads, 0, s>>>(gy, n->wflip, nullptr, g2, D, H, W, 0);
  k_relu_back<<<512, 256, 0, s>>>(g2, z2, (size_t)B * kC2 * vol);
  // layer 2
  k_conv_wgrad<kC2, kC3><<<g, kConvThreads, 0, s>>>(z1, g2, n->part, D, H, W, 1);
  k_wgrad_reduce<<<64, 256, 0, s>>>(n->part, B * nblk, kW2 + kC3, n->grads + kOffW2, n->grads + kOffB2, kW2);
  k_flip_weights<<<32, 256, 0, s>>>(P + kOffW2, n->wflip, kC2, kC3);
  k_conv_fwd<kC3, kC2><<<g, kConvThreads, 0, s>>>(g2, n->wflip, nullptr, g1, D, H, W, 0);
  k_relu_back<<<512, 256, 0, s>>>(g1, z1, (size_t)B * kC2 * vol);
  // layer 1
  k_conv_wgrad<kC1, kC2><<<g, kConvThreads, 0, s>>>(x, g1, n->part, D, H, W, 0);
  k_wgrad_reduce<<<64, 256, 0, s>>>(n->part, B * nblk, kW1 + kC2, n->grads + kOffW1, n->grads + kOffB1, kW1);
  return ncuda(n, cudaGetLastError(), "network backward");
}

}  // namespace

extern "C" {

int rsx_net_create(rsx_net** out, int device) {
  if (!out) return RSX_EINVAL;
  *out = nullptr;
  if (cudaSetDevice(device) != cudaSuccess) {
    cudaGetLastError();
    return RSX_ECUDA;
  }
  rsx_net* n = new rsx_net();
  n->device = device;
  if (cudaMalloc(&n->params, kNParams * sizeof(float)) != cudaSuccess ||
      cudaMalloc(&n->grads, kNParams * sizeof(float)) != cudaSuccess ||
      cudaMalloc(&n->adam_m, kNParams * sizeof(float)) != cudaSuccess ||
      cudaMalloc(&n->adam_v, kNParams * sizeof(float)) != cudaSuccess ||
      cudaMalloc(&n->wflip, kW2 * sizeof(float)) != cudaSuccess || cudaMalloc(&n->loss, sizeof(double)) != cudaSuccess) {
    cudaGetLastError();
    rsx_net_destroy(n);
    return RSX_ENOMEM;
  }
  cudaMemset(n->params, 0, kNParams * sizeof(float));
  cudaMemset(n->adam_m, 0, kNParams * sizeof(float));
  cudaMemset(n->adam_v, 0, kNParams * sizeof(float));
  *out = n;
  return RSX_OK;
}

int rsx_net_param_count(void) { return kNParams; }

int rsx_net_set_params(rsx_net* n, const float* host, int count) {
  if (!n || !host || count != kNParams) return RSX_EINVAL;
  cudaSetDevice(n->device);
  n->step = 0;
  cudaMemset(n->adam_m, 0, kNParams * sizeof(float));
  cudaMemset(n->adam_v, 0, kNParams * sizeof(float));
  return ncuda(n, cudaMemcpy(n->params, host, kNParams * sizeof(float), cudaMemcpyHostToDevice), "set params");
}

int rsx_net_get_params(rsx_net* n, float* host, int count) {
  if (!n || !host || count != kNParams) return RSX_EINVAL;
  cudaSetDevice(n->device);
  return ncuda(n, cudaMemcpy(host, n->params, kNParams * sizeof(float), cudaMemcpyDeviceToHost), "get params");
}

int rsx_net_forward(rsx_net* n, const float* x, int B, int D, int H, int W, float* out, void* stream) {
  if (!n || !x || !out || B < 1 || D < 1 || H < 1 || W < 1) return RSX_EINVAL;
  cudaSetDevice(n->device);
  return forward(n, x, B, D, H, W, out, (cudaStream_t)stream);
}

int rsx_net_loss_grad(rsx_net* n, const float* x, const float* target, int B, int D, int H, int W, int border,
                      double* loss_host, float* grad_host, void* stream) {
  if (!n || !x || !target || B < 1 || D <= 2 * border || H <= 2 * border || W <= 2 * border) return RSX_EINVAL;
  cudaSetDevice(n->device);
  cudaStream_t s = (cudaStream_t)stream;
  cudaMemsetAsync(n->loss, 0, sizeof(double), s);
  int rc = backward(n, x, target, B, D, H, W, border, s);
  if (rc) return rc;
  if (loss_host) rc = ncuda(n, cudaMemcpyAsync(loss_host, n->loss, sizeof(double), cudaMemcpyDeviceToHost, s), "loss");
  if (!rc && grad_host)
    rc = ncuda(n, cudaMemcpyAsync(grad_host, n->grads, kNParams * sizeof(float), cudaMemcpyDeviceToHost, s), "grads");
  if (!rc) rc = ncuda(n, cudaStreamSynchronize(s), "sync");
  return rc;
}

int rsx_net_train_step(rsx_net* n, const float* x, const float* target, int B, int D, int H, int W, int border,
                       float lr, double* loss_host, void* stream) {
  if (!n || !x || !target || B < 1 || D <= 2 * border || H <= 2 * border || W <= 2 * border || !(lr > 0.f))
    return RSX_EINVAL;
  cudaSetDevice(n->device);
  cudaStream_t s = (cudaStream_t)stream;
  cudaMemsetAsync(n->loss, 0, sizeof(double), s);
  int rc = backward(n, x, target, B, D, H, W, border, s);
  if (rc) return rc;
  ++n->step;
  const float b1 = 0.9f, b2 = 0.999f;
  const float c1 = 1.f - powf(b1, (float)n->step), c2 = 1.f - powf(b2, (float)n->step);
  k_adam<<<(kNParams + 255) / 256, 256, 0, s>>>(n->params, n->grads, n->adam_m, n->adam_v, kNParams, lr, b1, b2, 1e-8f,
                                                 c1, c2);
  rc = ncuda(n, cudaGetLastError(), "adam");
  if (!rc && loss_host)
    rc = ncuda(n, cudaMemcpyAsync(loss_host, n->loss, sizeof(double), cudaMemcpyDeviceToHost, s), "loss");
  return rc;
}

const char* rsx_net_last_error(const rsx_net* n) { return n ? n->err : "null network"; }

int rsx_net_destroy(rsx_net* n) {
  if (!n) return RSX_OK;
  cudaSetDevice(n->device);
  cudaDeviceSynchronize();
  void* bufs[] = {n->params, n->grads, n->adam_m, n->adam_v, n->wflip, n->act, n->gout, n->part, n->loss};
  for (void* p : bufs)
    if (p) cudaFree(p);
  delete n;
  return RSX_OK;
}

}  // extern "C"
