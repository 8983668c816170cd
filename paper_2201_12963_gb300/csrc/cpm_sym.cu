// S-apply from symmetric packed storage (mixed precision, one replica): q = S (b + dpsi v) with
// S = O A^-1 (Eqs. 8-9) or, per mirror block of the doubled cell, the block's projected inverse
// (Eqs. 13-15).
//
// S (or each mirror block S+-) is symmetric, so only its upper triangle of 128 x 128 tiles is kept:
// tile (I, J), I <= J, at packed index I nt - I (I - 1) / 2 + (J - I), each tile row-major
// (diagonal tiles in full).  One read of an off-diagonal tile serves both S_IJ x_J (rows of block I)
// and S_IJ^T x_I (rows of block J), so the HBM bytes per step are about half of the full matrix.
// Each tile's 128 row products and 128 transposed products are added into a float64 row vector
// (qpart, shared with the streaming variant) with atomics, nt additions per row from different
// CTAs; k_sapply_finish then forms q_raw = qpart + dpsi S v with the projection sums and clears
// qpart for the next call.
#include "cpm_internal.cuh"

#include <algorithm>

namespace cpm {

constexpr int SY_T = 128;                 // tile edge
constexpr int SY_THREADS = 256;           // 8 warps: warp g streams rows 16 g .. 16 g + 15 of a tile
constexpr int SY_SMEM_MAX = 220 * 1024;

__host__ __device__ __forceinline__ long long sy_tiles(int nt) { return (long long)nt * (nt + 1) / 2; }

// Packed tiles of the float32 copy from the float64 master (rows of stride ld; zero beyond n).
__global__ void __launch_bounds__(256) k_pack_sym(const double* __restrict__ S, int n, int ld, int nt,
                                                  float* __restrict__ Sp) {
  const int J = blockIdx.x, I = blockIdx.y;
  if (J < I) return;
  const long long t = (long long)I * nt - (long long)I * (I - 1) / 2 + (J - I);
  float* tile = Sp + t * SY_T * SY_T;
  for (int e = threadIdx.x; e < SY_T * SY_T; e += blockDim.x) {
    const int r = I * SY_T + e / SY_T, c = J * SY_T + e % SY_T;
    tile[e] = (r < n && c < n) ? (float)S[(size_t)r * ld + c] : 0.0f;
  }
}

// Persistent streaming over the packed tiles: each CTA takes an equal contiguous range of tiles,
// with the next tile's 16 loads per thread in flight while the current one is reduced.
__global__ void __launch_bounds__(SY_THREADS, 1) k_sapply_sym(const float* __restrict__ Sp, int nt, int n,
                                                             const float* __restrict__ xh,
                                                             const float* __restrict__ xl, double* __restrict__ qpart,
                                                             int npad) {
  pdl_enter();
  extern __shared__ __align__(16) float sy_sm[];
  float* sxh = sy_sm;                        // [npad]
  float* sxl = sxh + npad;                   // [npad]
  float* R = sxl + npad;                     // [128][33] per-lane row contributions
  float* C = R + SY_T * 33;                  // [8][128] per-warp column contributions
  const int tid = threadIdx.x, q = tid & 31, g = tid >> 5;
  for (int i = tid; i < npad; i += SY_THREADS) {
    sxh[i] = i < n ? xh[i] : 0.f;
    sxl[i] = i < n ? xl[i] : 0.f;
  }
  __syncthreads();
  const long long total = sy_tiles(nt);
  const long long per = (total + gridDim.x - 1) / gridDim.x;
  long long t = blockIdx.x * per;
  const long long tend = min(total, t + per);
  if (t >= tend) return;
  int I = 0;
  long long base = 0, rowlen = nt;
  while (t >= base + rowlen) {
    base += rowlen;
    ++I;
    --rowlen;
  }
  int J = I + (int)(t - base);
  const float4* S4 = reinterpret_cast<const float4*>(Sp);
  float4 cur[16], nxt[16];
#pragma unroll
  for (int k = 0; k < 16; ++k) cur[k] = __ldcs(S4 + t * (SY_T * SY_T / 4) + (g * 16 + k) * 32 + q);
  const float4* xh4 = reinterpret_cast<const float4*>(sxh);
  const float4* xl4 = reinterpret_cast<const float4*>(sxl);
  while (t < tend) {
    const long long tn = t + 1;
    int In = I, Jn = J + 1;
    if (Jn == nt) {
      In = I + 1;
      Jn = In;
    }
    if (tn < tend) {
#pragma unroll
      for (int k = 0; k < 16; ++k) nxt[k] = __ldcs(S4 + tn * (SY_T * SY_T / 4) + (g * 16 + k) * 32 + q);
    }
    const float4 xjh = xh4[J * 32 + q], xjl = xl4[J * 32 + q];
    float4 ch = make_float4(0.f, 0.f, 0.f, 0.f), cl = ch;
#pragma unroll
    for (int k = 0; k < 16; ++k) {
      const int r = g * 16 + k;
      const float4 s = cur[k];
      const float rh = s.x * xjh.x + s.y * xjh.y + s.z * xjh.z + s.w * xjh.w;
      const float rl = s.x * xjl.x + s.y * xjl.y + s.z * xjl.z + s.w * xjl.w;
      R[r * 33 + q] = rh + rl;
      const float xr = sxh[I * SY_T + r], xrl = sxl[I * SY_T + r];
      ch.x = fmaf(s.x, xr, ch.x);
      ch.y = fmaf(s.y, xr, ch.y);
      ch.z = fmaf(s.z, xr, ch.z);
      ch.w = fmaf(s.w, xr, ch.w);
      cl.x = fmaf(s.x, xrl, cl.x);
      cl.y = fmaf(s.y, xrl, cl.y);
      cl.z = fmaf(s.z, xrl, cl.z);
      cl.w = fmaf(s.w, xrl, cl.w);
    }
    float* cw = C + g * SY_T + 4 * q;
    cw[0] = ch.x + cl.x;
    cw[1] = ch.y + cl.y;
    cw[2] = ch.z + cl.z;
    cw[3] = ch.w + cl.w;
    __syncthreads();
    if (tid < SY_T) {
      Acc<float> a;
      for (int l = 0; l < 32; ++l) a.add(R[tid * 33 + l]);
      const int row = I * SY_T + tid;
      if (row < n) atomicAdd(&qpart[row], a.value());
      if (I != J) {
        Acc<float> b;
        for (int w = 0; w < SY_THREADS / 32; ++w) b.add(C[w * SY_T + tid]);
        const int col = J * SY_T + tid;
        if (col < n) atomicAdd(&qpart[col], b.value());
      }
    }
    __syncthreads();
    if (tn < tend) {
#pragma unroll
      for (int k = 0; k < 16; ++k) cur[k] = nxt[k];
    }
    t = tn;
    I = In;
    J = Jn;
  }
}

static size_t sym_smem(int npad) { return sizeof(float) * (2 * (size_t)npad + SY_T * 33 + 8 * SY_T); }

// The same packed S-apply with the tiles moved into shared memory by bulk asynchronous copies
// (cp.async.bulk, completion on an mbarrier per stage): SYT_STAGES tiles of 64 KB are requested
// at once, so a CTA with few tiles (the paper-scale cell: two) has all its bytes in flight from
// the start, and a CTA with many streams them through the stages.  The right-hand side is read
// per tile (the x slices of the tile's row and column blocks, prefetched one tile ahead), so the
// variant has no limit on n from shared memory.  Every wait is bounded: on a timeout the CTA
// records CPM's timeout status, waits (bounded) for its copies still in flight and returns.
constexpr int SYT_STAGES = 3;
constexpr long long SYT_WAIT_LIMIT = 1LL << 22;      // mbarrier polls (32 ns sleeps) per wait
constexpr uint32_t SYT_TILE_BYTES = SY_T * SY_T * sizeof(float);

__device__ __forceinline__ uint32_t syt_smem(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }

__device__ __forceinline__ void syt_issue(uint64_t* mbar, float* dst, const float* src) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(syt_smem(mbar)), "r"(SYT_TILE_BYTES)
               : "memory");
  asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
                   syt_smem(dst)),
               "l"(src), "r"(SYT_TILE_BYTES), "r"(syt_smem(mbar))
               : "memory");
}

// true once the phase `parity` of the mbarrier has completed, polling at most `limit` times
__device__ __forceinline__ bool syt_wait(uint64_t* mbar, uint32_t parity, long long limit) {
  uint32_t done = 0;
  for (long long it = 0; it < limit && !done; ++it) {
    asm volatile("{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}"
                 : "=r"(done)
                 : "r"(syt_smem(mbar)), "r"(parity)
                 : "memory");
    if (!done) __nanosleep(32);
  }
  return done != 0;
}

__global__ void __launch_bounds__(SY_THREADS, 1) k_sapply_sym_tma(const float* __restrict__ Sp, int nt, int n,
                                                                 const float* __restrict__ xh,
                                                                 const float* __restrict__ xl,
                                                                 double* __restrict__ qpart, int short_wait,
                                                                 int* __restrict__ status) {
  extern __shared__ __align__(128) float syt_sm[];
  float* tiles = syt_sm;                               // [SYT_STAGES][128 * 128]
  float* R = tiles + SYT_STAGES * SY_T * SY_T;         // [128][33] per-lane row contributions
  float* C = R + SY_T * 33;                            // [8][128] per-warp column contributions
  float* X = C + 8 * SY_T;                             // [2][4][128] x slices: I hi, I lo, J hi, J lo
  uint64_t* mbar = reinterpret_cast<uint64_t*>(X + 2 * 4 * SY_T);   // [SYT_STAGES]
  __shared__ int ok_sh;
  const int tid = threadIdx.x, q = tid & 31, g = tid >> 5;
  const long long total = sy_tiles(nt);
  const long long per = (total + gridDim.x - 1) / gridDim.x;
  const long long t0 = blockIdx.x * per;
  const long long t1 = min(total, t0 + per);
  if (t0 >= t1) return;
  int I = 0;
  long long base = 0, rowlen = nt;
  while (t0 >= base + rowlen) {
    base += rowlen;
    ++I;
    --rowlen;
  }
  int J = I + (int)(t0 - base);
  if (tid == 0) {
    for (int k = 0; k < SYT_STAGES; ++k)
      asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(syt_smem(&mbar[k])), "r"(1) : "memory");
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    ok_sh = 1;
  }
  __syncthreads();
  // the packed tiles are written when the context is built, never by the step: their copies start
  // before the wait for the preceding kernels
  if (tid == 0)
    for (int k = 0; k < SYT_STAGES && t0 + k < t1; ++k)
      syt_issue(&mbar[k], tiles + (size_t)k * SY_T * SY_T, Sp + (t0 + k) * (long long)(SY_T * SY_T));
  pdl_enter();                                         // x (and qpart) come from the preceding kernels
  // x slices of tile (I, J): threads 0..127 the row block I, 128..255 the column block J
  const int xi = tid & (SY_T - 1), xs = tid >> 7;      // xs: 0 = I, 1 = J
  {
    const int idx = (xs ? J : I) * SY_T + xi;
    X[(2 * xs) * SY_T + xi] = idx < n ? xh[idx] : 0.f;
    X[(2 * xs + 1) * SY_T + xi] = idx < n ? xl[idx] : 0.f;
  }
  __syncthreads();
  long long k = 0;
  for (long long t = t0; t < t1; ++t, ++k) {
    const int st = (int)(k % SYT_STAGES), xb = (int)(k & 1);
    const uint32_t parity = (uint32_t)((k / SYT_STAGES) & 1);
    int In = I, Jn = J + 1;
    if (Jn == nt) {
      In = I + 1;
      Jn = In;
    }
    // the next tile's x slices, into registers
    float nh = 0.f, nl = 0.f;
    if (t + 1 < t1) {
      const int idx = (xs ? Jn : In) * SY_T + xi;
      if (idx < n) {
        nh = xh[idx];
        nl = xl[idx];
      }
    }
    if (tid == 0) {
      const bool got = syt_wait(&mbar[st], parity, (short_wait && k == 0) ? 0 : SYT_WAIT_LIMIT);
      if (!got) {
        latch_error(status, DE_TIMEOUT);
        // copies issued and not yet consumed: tiles k .. min(k + SYT_STAGES, count) - 1
        for (long long m = k; m < k + SYT_STAGES && t0 + m < t1; ++m)
          syt_wait(&mbar[m % SYT_STAGES], (uint32_t)((m / SYT_STAGES) & 1), SYT_WAIT_LIMIT);
        ok_sh = 0;
      }
    }
    __syncthreads();
    if (!ok_sh) return;
    const float4* T4 = reinterpret_cast<const float4*>(tiles + (size_t)st * SY_T * SY_T);
    const float* Xb = X + xb * 4 * SY_T;
    const float4 xjh = reinterpret_cast<const float4*>(Xb + 2 * SY_T)[q];
    const float4 xjl = reinterpret_cast<const float4*>(Xb + 3 * SY_T)[q];
    float4 ch = make_float4(0.f, 0.f, 0.f, 0.f), cl = ch;
#pragma unroll
    for (int kk = 0; kk < 16; ++kk) {
      const int r = g * 16 + kk;
      const float4 s4 = T4[r * 32 + q];
      const float rh = s4.x * xjh.x + s4.y * xjh.y + s4.z * xjh.z + s4.w * xjh.w;
      const float rl = s4.x * xjl.x + s4.y * xjl.y + s4.z * xjl.z + s4.w * xjl.w;
      R[r * 33 + q] = rh + rl;
      const float xr = Xb[r], xrl = Xb[SY_T + r];
      ch.x = fmaf(s4.x, xr, ch.x);
      ch.y = fmaf(s4.y, xr, ch.y);
      ch.z = fmaf(s4.z, xr, ch.z);
      ch.w = fmaf(s4.w, xr, ch.w);
      cl.x = fmaf(s4.x, xrl, cl.x);
      cl.y = fmaf(s4.y, xrl, cl.y);
      cl.z = fmaf(s4.z, xrl, cl.z);
      cl.w = fmaf(s4.w, xrl, cl.w);
    }
    float* cw = C + g * SY_T + 4 * q;
    cw[0] = ch.x + cl.x;
    cw[1] = ch.y + cl.y;
    cw[2] = ch.z + cl.z;
    cw[3] = ch.w + cl.w;
    __syncthreads();                                   // the stage is read: refill it
    if (tid == 0 && t + SYT_STAGES < t1) {
      asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
      syt_issue(&mbar[st], tiles + (size_t)st * SY_T * SY_T, Sp + (t + SYT_STAGES) * (long long)(SY_T * SY_T));
    }
    if (tid < SY_T) {
      Acc<float> a;
      for (int l = 0; l < 32; ++l) a.add(R[tid * 33 + l]);
      const int row = I * SY_T + tid;
      if (row < n) atomicAdd(&qpart[row], a.value());
      if (I != J) {
        Acc<float> b;
        for (int w = 0; w < SY_THREADS / 32; ++w) b.add(C[w * SY_T + tid]);
        const int col = J * SY_T + tid;
        if (col < n) atomicAdd(&qpart[col], b.value());
      }
    }
    X[(xb ^ 1) * 4 * SY_T + (2 * xs) * SY_T + xi] = nh;
    X[(xb ^ 1) * 4 * SY_T + (2 * xs + 1) * SY_T + xi] = nl;
    __syncthreads();
    I = In;
    J = Jn;
  }
}

static size_t sym_tma_smem() {
  return sizeof(float) * ((size_t)SYT_STAGES * SY_T * SY_T + SY_T * 33 + 8 * SY_T + 2 * 4 * SY_T) +
         sizeof(uint64_t) * SYT_STAGES;
}

}  // namespace cpm

using namespace cpm;

// Packed upper-triangle tiles of S (or of both mirror blocks) from the float64 master.  Leaves
// c->sym_ok false when the right-hand side does not fit shared memory.
int cpm_internal_sym_setup(cpm_ctx* c) {
  c->sym_ok = false;
  if (!c->mixed) return CPM_OK;
  const int n = c->mirror ? c->nh : c->ne;
  const int nt = (n + SY_T - 1) / SY_T;
  const int npad = nt * SY_T;
  if (sym_smem(npad) > (size_t)SY_SMEM_MAX) return CPM_OK;
  if (!c->qpart) return CPM_OK;                // the float64 row accumulator of the streaming variant
  const int blocks = c->mirror ? 2 : 1;
  const long long tiles = sy_tiles(nt);
  CPM_CUDA(cudaMalloc(&c->sym_S, sizeof(float) * (size_t)blocks * tiles * SY_T * SY_T));
  for (int blk = 0; blk < blocks; ++blk) {
    const double* S = c->S64 + (size_t)blk * n * c->ld64;
    k_pack_sym<<<dim3(nt, nt), 256>>>(S, n, c->ld64, nt, c->sym_S + (size_t)blk * tiles * SY_T * SY_T);
    CPM_LAUNCH();
  }
  CPM_CUDA(cudaDeviceSynchronize());
  CPM_CUDA(cudaFuncSetAttribute(k_sapply_sym, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sym_smem(npad)));
  CPM_CUDA(cudaFuncSetAttribute(k_sapply_sym_tma, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sym_tma_smem()));
  c->sym_nt = nt;
  c->sym_ok = true;
  return CPM_OK;
}

// One S-apply of block blk (0, or 1 for the S- mirror block) from the packed tiles, then its finish.
int cpm_internal_sapply_sym(cpm_ctx* c, int blk, const float* xh, const float* xl, const double* b,
                            const double* dpsi, const double* Sv, const double* W, const double* c1, double* qout,
                            cudaStream_t st) {
  const int n = c->mirror ? c->nh : c->ne;
  const int nt = c->sym_nt, npad = nt * SY_T;
  const float* Sp = c->sym_S + (size_t)blk * sy_tiles(nt) * SY_T * SY_T;
  double* qpart = c->qpart + (size_t)blk * n;
  if (c->sapply_variant == CPM_SAPPLY_SYM_TMA)
    CPM_CUDA(launch_pdl(k_sapply_sym_tma, c->n_sm, SY_THREADS, sym_tma_smem(), st, Sp, nt, n, xh, xl, qpart,
                        c->wait_test ? 1 : 0, c->status));
  else
    CPM_CUDA(launch_pdl(k_sapply_sym, c->n_sm, SY_THREADS, sym_smem(npad), st, Sp, nt, n, xh, xl, qpart, npad));
  ++c->launches;
  CPM_LAUNCH();
  CPM_CUDA(launch_pdl(k_sapply_finish, (n + FIN_THREADS - 1) / FIN_THREADS, FIN_THREADS, 0, st, n, qpart, b, dpsi, Sv, W, c1, qout, c->scal));
  ++c->launches;
  CPM_LAUNCH();
  return CPM_OK;
}
