// SPME convolution (the reciprocal-space part of the Ewald sums behind Eq. 3, Sec. II.B) on the
// mesh in float32 without the FFT library: forward 3-D real-to-complex
// transform, multiplication by the influence function G (with the reciprocal energy), inverse
// transform, as five launches that each keep their lines in shared memory:
//   z: real-to-complex per mesh line (warp per line)
//   y: complex transform of every (x, k_z) column (block per tile of 32 contiguous columns)
//   x: forward transform, times G (+ energy), inverse transform, in one kernel per column tile
//   y: inverse
//   z: complex-to-real per line (Hermitian completion of the half spectrum)
// Each line transform of length n = n1 n2 is the four-step decomposition of the discrete Fourier
// transform: n1 transforms of length n2 over the strided subsequences, twiddle factors
// w_n^(j1 k2), then n2 transforms of length n1; the short transforms are direct sums with the
// per-axis table w_n^t = exp(-2 pi i t / n) (computed in float64 on the host).  Unnormalised like
// the library transforms, so the influence function is shared with the cuFFT path.
#include "cpm_internal.cuh"

#include <algorithm>
#include <cmath>
#include <vector>

namespace cpm {

constexpr int FZ_WARPS = 4;          // lines per block of the z passes
constexpr int FC_THREADS = 256;      // column-pass block: 32 columns x 8 threads per column
constexpr int FC_COLS = 32;

struct FftAxis {
  int K, n1, n2;
  const float2* tw;                  // [K] exp(-2 pi i t / K)
};

__device__ __forceinline__ float2 twid(const float2* tw, int t, bool inv) {
  const float2 w = tw[t];
  return inv ? make_float2(w.x, -w.y) : w;
}
__device__ __forceinline__ float2 cfma(float2 a, float2 w, float2 acc) {
  acc.x = fmaf(a.x, w.x, fmaf(-a.y, w.y, acc.x));
  acc.y = fmaf(a.x, w.y, fmaf(a.y, w.x, acc.y));
  return acc;
}
__device__ __forceinline__ float2 cmul(float2 a, float2 w) { return cfma(a, w, make_float2(0.f, 0.f)); }

// Four-step stage A for output o = j1 n2 + k2 of one line held at x[j * xs] (shared memory):
// sum_j2 x[j1 + n1 j2] w_n2^(j2 k2), times w_n^(j1 k2).
__device__ __forceinline__ float2 stage_a(const float2* x, int xs, int o, const FftAxis& a, bool inv) {
  const int j1 = o / a.n2, k2 = o - j1 * a.n2;
  float2 acc = make_float2(0.f, 0.f);
  int t = 0;
  for (int j2 = 0; j2 < a.n2; ++j2) {
    acc = cfma(x[(j1 + a.n1 * j2) * xs], twid(a.tw, t * a.n1, inv), acc);
    t += k2;
    if (t >= a.n2) t -= a.n2;
  }
  return cmul(acc, twid(a.tw, (j1 * k2) % a.K, inv));
}

// Four-step stage C for output k = k2 + n2 k1: sum_j1 y[j1 n2 + k2] w_n1^(j1 k1).
__device__ __forceinline__ float2 stage_c(const float2* y, int ys, int k, const FftAxis& a, bool inv) {
  const int k1 = k / a.n2, k2 = k - k1 * a.n2;
  float2 acc = make_float2(0.f, 0.f);
  int t = 0;
  for (int j1 = 0; j1 < a.n1; ++j1) {
    acc = cfma(y[(j1 * a.n2 + k2) * ys], twid(a.tw, t * a.n2, inv), acc);
    t += k1;
    if (t >= a.n1) t -= a.n1;
  }
  return acc;
}

// z pass, forward: real line (K3 floats) -> K3/2 + 1 complex outputs.  One warp per line.
__global__ void __launch_bounds__(FZ_WARPS * 32) k_fftz_r2c(const float* __restrict__ mesh, float2* __restrict__ spec,
                                                            int nlines, long long Mr_s, long long Mc_s, FftAxis az) {
  extern __shared__ float2 fz_sm[];
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  const int K = az.K, Kh = K / 2 + 1;
  float2* x = fz_sm + (size_t)w * 2 * K;
  float2* y = x + K;
  float2* stw = fz_sm + (size_t)FZ_WARPS * 2 * K;          // twiddle table, shared by the block
  for (int t = threadIdx.x; t < K; t += blockDim.x) stw[t] = az.tw[t];
  __syncthreads();
  az.tw = stw;
  const int line = blockIdx.x * FZ_WARPS + w;
  if (line >= nlines) return;
  const float* src = mesh + (size_t)blockIdx.y * Mr_s + (size_t)line * K;
  for (int j = lane; j < K; j += 32) x[j] = make_float2(src[j], 0.f);
  __syncwarp();
  for (int o = lane; o < K; o += 32) y[o] = stage_a(x, 1, o, az, false);
  __syncwarp();
  float2* dst = spec + (size_t)blockIdx.y * Mc_s + (size_t)line * Kh;
  for (int k = lane; k < Kh; k += 32) dst[k] = stage_c(y, 1, k, az, false);
}

// z pass, inverse: K3/2 + 1 complex (Hermitian half) -> K3 real outputs.
__global__ void __launch_bounds__(FZ_WARPS * 32) k_fftz_c2r(const float2* __restrict__ spec, float* __restrict__ phi,
                                                            int nlines, long long Mr_s, long long Mc_s, FftAxis az) {
  extern __shared__ float2 fz_sm[];
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  const int K = az.K, Kh = K / 2 + 1;
  float2* x = fz_sm + (size_t)w * 2 * K;
  float2* y = x + K;
  float2* stw = fz_sm + (size_t)FZ_WARPS * 2 * K;          // twiddle table, shared by the block
  for (int t = threadIdx.x; t < K; t += blockDim.x) stw[t] = az.tw[t];
  __syncthreads();
  az.tw = stw;
  const int line = blockIdx.x * FZ_WARPS + w;
  if (line >= nlines) return;
  const float2* src = spec + (size_t)blockIdx.y * Mc_s + (size_t)line * Kh;
  for (int k = lane; k < K; k += 32) {
    if (k < Kh) {
      x[k] = src[k];
    } else {
      const float2 v = src[K - k];
      x[k] = make_float2(v.x, -v.y);
    }
  }
  __syncwarp();
  for (int o = lane; o < K; o += 32) y[o] = stage_a(x, 1, o, az, true);
  __syncwarp();
  float* dst = phi + (size_t)blockIdx.y * Mr_s + (size_t)line * K;
  for (int k = lane; k < K; k += 32) dst[k] = stage_c(y, 1, k, az, true).x;
}

// Column passes over spec viewed as [A][K][B] (transform along K; B contiguous): one block per
// (tile of 32 contiguous b, a, replica).  CONV (the x pass, A = 1): forward, times G[k B + b] with
// the reciprocal energy 1/2 sum_full G |rho^|^2 accumulated into scal[energy_slot] (if >= 0),
// inverse.  Otherwise one transform in the direction `inv`.
template <bool CONV>
__global__ void __launch_bounds__(FC_THREADS) k_fft_cols(float2* __restrict__ spec, long long Mc_s, int B, FftAxis ax,
                                                         bool inv, const float* __restrict__ G, int K3, int K3h,
                                                         int energy_slot, double* __restrict__ scal) {
  extern __shared__ float2 fc_sm[];
  const int K = ax.K;
  float2* b0 = fc_sm;                      // [K][32]
  float2* b1 = fc_sm + (size_t)K * FC_COLS;
  float2* stw = b1 + (size_t)K * FC_COLS;  // twiddle table
  for (int t = threadIdx.x; t < K; t += blockDim.x) stw[t] = ax.tw[t];
  ax.tw = stw;
  const int c = threadIdx.x & (FC_COLS - 1), r = threadIdx.x / FC_COLS, nr = FC_THREADS / FC_COLS;
  const int bcol = blockIdx.x * FC_COLS + c;
  const bool live = bcol < B;
  float2* base = spec + (size_t)blockIdx.z * Mc_s + (size_t)blockIdx.y * K * B;
  for (int k = r; k < K; k += nr) b0[k * FC_COLS + c] = live ? base[(size_t)k * B + bcol] : make_float2(0.f, 0.f);
  __syncthreads();
  const int passes = CONV ? 2 : 1;
  Acc<float> e;
  for (int pass = 0; pass < passes; ++pass) {
    const bool dir = CONV ? (pass == 1) : inv;
    for (int o = r; o < K; o += nr) b1[o * FC_COLS + c] = stage_a(b0 + c, FC_COLS, o, ax, dir);
    __syncthreads();
    for (int k = r; k < K; k += nr) b0[k * FC_COLS + c] = stage_c(b1 + c, FC_COLS, k, ax, dir);
    __syncthreads();
    if (CONV && pass == 0) {
      for (int k = r; k < K; k += nr) {
        float2 v = b0[k * FC_COLS + c];
        const float g = live ? G[(size_t)k * B + bcol] : 0.f;
        if (energy_slot >= 0) {
          const int kz = bcol % K3h;
          const float wgt = (kz == 0 || 2 * kz == K3) ? 0.5f : 1.0f;
          e.add(wgt * g * (v.x * v.x + v.y * v.y));
        }
        v.x *= g;
        v.y *= g;
        b0[k * FC_COLS + c] = v;
      }
      __syncthreads();
    }
  }
  if (live)
    for (int k = r; k < K; k += nr) base[(size_t)k * B + bcol] = b0[k * FC_COLS + c];
  if (CONV && energy_slot >= 0) {
    e.warp_reduce();
    double acc[1] = {e.value()};
    double* const dst[1] = {scal + blockIdx.z * NSCAL + energy_slot};
    block_atomic_add<1>(acc, dst);
  }
}

static FftAxis axis(const cpm_ctx* c, int d) {
  FftAxis a;
  a.K = c->K[d];
  a.n1 = c->fft_n1[d];
  a.n2 = a.K / a.n1;
  a.tw = c->fft_tw + c->fft_tw_off[d];
  return a;
}

static size_t cols_smem(int K) { return sizeof(float2) * (2 * (size_t)K * FC_COLS + K); }
static size_t z_smem(int K) { return sizeof(float2) * (2 * (size_t)K * FZ_WARPS + K); }

}  // namespace cpm

using namespace cpm;

// Twiddle tables and factorisations; false (and the library transform stays in use) when a mesh
// axis is too long for the shared-memory column tiles.
int cpm_internal_fft_setup(cpm_ctx* c) {
  c->fft_own_ok = false;
  if (!c->mixed) return CPM_OK;
  int off = 0;
  std::vector<float2> tw;
  for (int d = 0; d < 3; ++d) {
    const int K = c->K[d];
    if (d < 2 && cols_smem(K) > 200 * 1024) return CPM_OK;
    int n1 = 1;
    for (int f = 1; f * f <= K; ++f)
      if (K % f == 0) n1 = f;
    c->fft_n1[d] = n1;
    c->fft_tw_off[d] = off;
    for (int t = 0; t < K; ++t) {
      const double ang = -2.0 * PI * (double)t / (double)K;
      tw.push_back(make_float2((float)std::cos(ang), (float)std::sin(ang)));
    }
    off += K;
  }
  if (z_smem(c->K[2]) > 200 * 1024) return CPM_OK;
  CPM_CUDA(cudaMalloc(&c->fft_tw, sizeof(float2) * tw.size()));
  CPM_CUDA(cudaMemcpy(c->fft_tw, tw.data(), sizeof(float2) * tw.size(), cudaMemcpyHostToDevice));
  const int zs = (int)z_smem(c->K[2]);
  const int cs = (int)std::max(cols_smem(c->K[0]), cols_smem(c->K[1]));
  CPM_CUDA(cudaFuncSetAttribute(k_fftz_r2c, cudaFuncAttributeMaxDynamicSharedMemorySize, zs));
  CPM_CUDA(cudaFuncSetAttribute(k_fftz_c2r, cudaFuncAttributeMaxDynamicSharedMemorySize, zs));
  CPM_CUDA(cudaFuncSetAttribute(k_fft_cols<true>, cudaFuncAttributeMaxDynamicSharedMemorySize, cs));
  CPM_CUDA(cudaFuncSetAttribute(k_fft_cols<false>, cudaFuncAttributeMaxDynamicSharedMemorySize, cs));
  c->fft_own_ok = true;
  return CPM_OK;
}

// mesh_r (charges) -> mesh_phi (potential), float32, nrep replicas; energy into scal[energy_slot]
// when energy_slot >= 0.  Counts its launches in c->launches.
int cpm_internal_convolve_own(cpm_ctx* c, int nrep, int energy_slot, cudaStream_t st) {
  const FftAxis ax = axis(c, 0), ay = axis(c, 1), az = axis(c, 2);
  const int K1 = c->K[0], K2 = c->K[1], K3 = c->K[2], K3h = K3 / 2 + 1;
  const int lines = K1 * K2;
  const size_t zs = z_smem(K3);
  float* mr = (float*)c->mesh_r;
  float2* mc = (float2*)c->mesh_c;
  float* mp = (float*)c->mesh_phi;
  const dim3 gz((lines + FZ_WARPS - 1) / FZ_WARPS, nrep);
  k_fftz_r2c<<<gz, FZ_WARPS * 32, zs, st>>>(mr, mc, lines, c->Mr_s, c->Mc_s, az);
  ++c->launches;
  CPM_LAUNCH();
  // y: spec as [K1][K2][K3h]
  const dim3 gy((K3h + FC_COLS - 1) / FC_COLS, K1, nrep);
  k_fft_cols<false><<<gy, FC_THREADS, cols_smem(K2), st>>>(mc, c->Mc_s, K3h, ay, false, nullptr, K3, K3h, -1, c->scal);
  ++c->launches;
  CPM_LAUNCH();
  // x with the influence function: spec as [1][K1][K2 K3h]
  const int Bx = K2 * K3h;
  const dim3 gx((Bx + FC_COLS - 1) / FC_COLS, 1, nrep);
  k_fft_cols<true><<<gx, FC_THREADS, cols_smem(K1), st>>>(mc, c->Mc_s, Bx, ax, false, c->G32, K3, K3h, energy_slot,
                                                           c->scal);
  ++c->launches;
  CPM_LAUNCH();
  k_fft_cols<false><<<gy, FC_THREADS, cols_smem(K2), st>>>(mc, c->Mc_s, K3h, ay, true, nullptr, K3, K3h, -1, c->scal);
  ++c->launches;
  CPM_LAUNCH();
  k_fftz_c2r<<<gz, FZ_WARPS * 32, zs, st>>>(mc, mp, lines, c->Mr_s, c->Mc_s, az);
  ++c->launches;
  CPM_LAUNCH();
  return CPM_OK;
}
