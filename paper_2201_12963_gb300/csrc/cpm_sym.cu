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
// CTAs.  The projection (Eq. 9) needs C^T q_raw and (A^-1 C)^T b of q_raw = qpart + dpsi S v.  With
// at most SY_FUSE_TILES_PER_CTA tiles per CTA the same kernel sums them (each tile's contributions
// as they are added into qpart, exactly, in fixed point; W^T b in one grid-strided pass at its
// start; the dpsi S v terms are dpsi times sums fixed at setup), and the projection reads qpart
// itself, adds dpsi S v and clears it for the next call; with more tiles per CTA k_sapply_finish
// forms q_raw and the sums in float64 and clears qpart.
#include "cpm_fixed.cuh"
#include "cpm_internal.cuh"

#include <algorithm>
#include <vector>

namespace cpm {

constexpr int SY_T = 128;                 // tile edge
constexpr int SY_THREADS = 256;           // 8 warps: warp g streams rows 16 g .. 16 g + 15 of a tile
constexpr int SY_SMEM_MAX = 220 * 1024;
constexpr int SY_FUSE_TILES_PER_CTA = 16;  // cpm_internal_sym_fuse: the largest tile count per CTA that fuses

__host__ __device__ __forceinline__ long long sy_tiles(int nt) { return (long long)nt * (nt + 1) / 2; }

// Inputs of the projection sums formed in the kernel and their destination.
struct SymSums {
  const float4* W32;     // A^-1 C of the block's rows split into float32 pairs: (W0 hi, W0 lo, W1 hi, W1 lo)
  const float* c1;       // second constraint column of the block's rows: an indicator (0 or 1)
  double* scal;          // S_CQ0, S_CQ1, S_WB0, S_WB1 accumulate here (null: no sums)
};

// Running sums of one thread: 1^T q_raw, c1^T q_raw, W_0^T b, W_1^T b, less the dpsi S v terms
// (constants times dpsi, added by the projection).  The S-apply products enter per tile as the
// float pairs of their compensated sums (the row's c1 weight prefetched a tile ahead); W^T b once
// per row in a grid-strided pass at the start of the kernel, from the float32 pair of the
// right-hand side (x hi + x lo) and of W, each product split exactly with fma.
struct SymAcc {
  Fx128 q0, q1, w0, w1;
  __device__ __forceinline__ void part(float vs, float vc, float c) {
    unsigned long long l0, h0, l1, h1;
    Fx128::image(vs, l0, h0);
    Fx128::image(vc, l1, h1);
    q0.add(l0, h0);
    q0.add(l1, h1);
    if (c != 0.f) {                                     // c1 is an indicator
      q1.add(l0, h0);
      q1.add(l1, h1);
    }
  }
  __device__ __forceinline__ void rows(const SymSums& f, const float* __restrict__ xh,
                                       const float* __restrict__ xl, int n) {
    for (int row = blockIdx.x * blockDim.x + threadIdx.x; row < n; row += gridDim.x * blockDim.x) {
      const float4 w = f.W32[row];
      const float bh = xh[row], bl = xl[row];
      const float p0 = w.x * bh, p1 = w.z * bh;
      w0.add(p0);
      w0.add(fmaf(w.x, bh, -p0) + (w.x * bl + w.y * bh));
      w1.add(p1);
      w1.add(fmaf(w.z, bh, -p1) + (w.z * bl + w.w * bh));
    }
  }
  // every thread of the block calls it
  __device__ __forceinline__ void flush(double* scal) {
    __shared__ Fx128 red[SY_THREADS / 32][4];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      q0.shfl_add(o);
      q1.shfl_add(o);
      w0.shfl_add(o);
      w1.shfl_add(o);
    }
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    if (lane == 0) {
      red[warp][0] = q0;
      red[warp][1] = q1;
      red[warp][2] = w0;
      red[warp][3] = w1;
    }
    __syncthreads();
    if (threadIdx.x < 4) {
      const int k = threadIdx.x;
      Fx128 a = red[0][k];
      for (int w = 1; w < SY_THREADS / 32; ++w) a.add(red[w][k]);
      const double v = a.value();
      const int dst = k == 0 ? S_CQ0 : k == 1 ? S_CQ1 : k == 2 ? S_WB0 : S_WB1;
      if (v != 0.0) atomicAdd(scal + dst, v);
    }
  }
};

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

// The c1 weight of the row (threads 0..127: row block I) or column (threads 128..255: column block
// J) whose products the thread adds in the epilogue of tile (I, J); 0 beyond n (loaded a tile
// ahead of its use).
__device__ __forceinline__ float sym_c1(const SymSums& fs, int I, int J, int n) {
  const int idx = ((threadIdx.x >> 7) ? J : I) * SY_T + (threadIdx.x & (SY_T - 1));
  return idx < n ? fs.c1[idx] : 0.f;
}

// Epilogue of tile (I, J), all threads: threads 0..127 reduce a row's 32 lane products, threads
// 128..255 (off the diagonal) a column's 8 warp products, in parallel; each result is added into
// qpart and, when fs.scal is set, into the projection sums (w: the row's or column's c1 weight).
__device__ __forceinline__ void sym_epilogue(const float* R, const float* C, int I, int J, int n,
                                             double* __restrict__ qpart, bool sums, float w, SymAcc& sa) {
  const int tid = threadIdx.x, r = tid & (SY_T - 1);
  Acc<float> a;
  int idx;
  if (tid < SY_T) {
    for (int l = 0; l < 32; ++l) a.add(R[r * 33 + l]);
    idx = I * SY_T + r;
  } else {
    if (I == J) return;
    for (int k = 0; k < SY_THREADS / 32; ++k) a.add(C[k * SY_T + r]);
    idx = J * SY_T + r;
  }
  if (idx < n) {
    atomicAdd(&qpart[idx], a.value());
    if (sums) sa.part(a.s, a.c, w);
  }
}

// Persistent streaming over the packed tiles: each CTA takes an equal contiguous range of tiles,
// with the next tile's 16 loads per thread in flight while the current one is reduced.
__global__ void __launch_bounds__(SY_THREADS, 1) k_sapply_sym(const float* __restrict__ Sp, int nt, int n,
                                                             const float* __restrict__ xh,
                                                             const float* __restrict__ xl, double* __restrict__ qpart,
                                                             int npad, SymSums fs) {
  extern __shared__ __align__(16) float sy_sm[];
  float* sxh = sy_sm;                        // [npad]
  float* sxl = sxh + npad;                   // [npad]
  float* R = sxl + npad;                     // [128][33] per-lane row contributions
  float* C = R + SY_T * 33;                  // [8][128] per-warp column contributions
  const int tid = threadIdx.x, q = tid & 31, g = tid >> 5;
  const long long total = sy_tiles(nt);
  const long long per = (total + gridDim.x - 1) / gridDim.x;
  long long t = blockIdx.x * per;
  const long long tend = min(total, t + per);
  const bool sums = fs.scal != nullptr;
  SymAcc sa;
  if (t >= tend) {
    pdl_enter();
    if (sums) {
      sa.rows(fs, xh, xl, n);
      sa.flush(fs.scal);
    }
    return;
  }
  int I = 0;
  long long base = 0, rowlen = nt;
  while (t >= base + rowlen) {
    base += rowlen;
    ++I;
    --rowlen;
  }
  int J = I + (int)(t - base);
  // the packed tiles are written when the context is built, never by the step: the first tile's
  // loads start before the wait for the preceding kernels and the staging of x
  const float4* S4 = reinterpret_cast<const float4*>(Sp);
  float4 cur[16], nxt[16];
#pragma unroll
  for (int k = 0; k < 16; ++k) cur[k] = __ldcs(S4 + t * (SY_T * SY_T / 4) + (g * 16 + k) * 32 + q);
  float wc = 0.f;
  if (sums) wc = sym_c1(fs, I, J, n);
  pdl_enter();
  for (int i = tid; i < npad; i += SY_THREADS) {
    sxh[i] = i < n ? xh[i] : 0.f;
    sxl[i] = i < n ? xl[i] : 0.f;
  }
  if (sums) sa.rows(fs, xh, xl, n);
  __syncthreads();
  const float4* xh4 = reinterpret_cast<const float4*>(sxh);
  const float4* xl4 = reinterpret_cast<const float4*>(sxl);
  while (t < tend) {
    const long long tn = t + 1;
    int In = I, Jn = J + 1;
    if (Jn == nt) {
      In = I + 1;
      Jn = In;
    }
    float wn = 0.f;
    if (tn < tend) {
#pragma unroll
      for (int k = 0; k < 16; ++k) nxt[k] = __ldcs(S4 + tn * (SY_T * SY_T / 4) + (g * 16 + k) * 32 + q);
      if (sums) wn = sym_c1(fs, In, Jn, n);
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
    sym_epilogue(R, C, I, J, n, qpart, sums, wc, sa);
    wc = wn;
    __syncthreads();
    if (tn < tend) {
#pragma unroll
      for (int k = 0; k < 16; ++k) cur[k] = nxt[k];
    }
    t = tn;
    I = In;
    J = Jn;
  }
  if (sums) sa.flush(fs.scal);
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
                                                                 int* __restrict__ status, SymSums fs) {
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
  const bool sums = fs.scal != nullptr;
  SymAcc sa;
  if (t0 >= t1) {
    pdl_enter();
    if (sums) {
      sa.rows(fs, xh, xl, n);
      sa.flush(fs.scal);
    }
    return;
  }
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
  float wc = 0.f;
  if (sums) wc = sym_c1(fs, I, J, n);
  pdl_enter();                                         // x (and qpart) come from the preceding kernels
  // x slices of tile (I, J): threads 0..127 the row block I, 128..255 the column block J
  const int xi = tid & (SY_T - 1), xs = tid >> 7;      // xs: 0 = I, 1 = J
  {
    const int idx = (xs ? J : I) * SY_T + xi;
    X[(2 * xs) * SY_T + xi] = idx < n ? xh[idx] : 0.f;
    X[(2 * xs + 1) * SY_T + xi] = idx < n ? xl[idx] : 0.f;
  }
  if (sums) sa.rows(fs, xh, xl, n);
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
    float wn = 0.f;
    if (t + 1 < t1) {
      const int idx = (xs ? Jn : In) * SY_T + xi;
      if (idx < n) {
        nh = xh[idx];
        nl = xl[idx];
        if (sums) wn = fs.c1[idx];
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
    sym_epilogue(R, C, I, J, n, qpart, sums, wc, sa);
    wc = wn;
    X[(xb ^ 1) * 4 * SY_T + (2 * xs) * SY_T + xi] = nh;
    X[(xb ^ 1) * 4 * SY_T + (2 * xs + 1) * SY_T + xi] = nl;
    __syncthreads();
    I = In;
    J = Jn;
  }
  if (sums) sa.flush(fs.scal);
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
  // the projection sums' inputs, per row of the blocks: W as float32 pairs, the c1 indicator,
  // and the dpsi S v sums
  const size_t rows = (size_t)blocks * n;
  std::vector<double> Wh(2 * rows), c1h(rows), svh(rows);
  CPM_CUDA(cudaMemcpy(Wh.data(), c->W, sizeof(double) * 2 * rows, cudaMemcpyDeviceToHost));
  CPM_CUDA(cudaMemcpy(c1h.data(), c->mirror ? c->e_c1m : c->e_c1, sizeof(double) * rows, cudaMemcpyDeviceToHost));
  CPM_CUDA(cudaMemcpy(svh.data(), c->Sv, sizeof(double) * rows, cudaMemcpyDeviceToHost));
  std::vector<float4> w32(rows);
  std::vector<float> c1f(rows);
  c->sym_sv[0] = c->sym_sv[1] = 0.0;
  bool indicator = true;                        // the kernel's sums take c1 as an indicator
  for (size_t r = 0; r < rows; ++r) {
    const double a = Wh[2 * r], b = Wh[2 * r + 1];
    const float ah = (float)a, bh = (float)b;
    w32[r] = make_float4(ah, (float)(a - (double)ah), bh, (float)(b - (double)bh));
    indicator = indicator && (c1h[r] == 0.0 || c1h[r] == 1.0);
    c1f[r] = (float)c1h[r];
    c->sym_sv[0] += svh[r];
    c->sym_sv[1] += c1h[r] * svh[r];
  }
  if (indicator) {                              // else the finish pass forms the sums (sym_w32 null)
    CPM_CUDA(cudaMalloc(&c->sym_w32, sizeof(float4) * rows));
    CPM_CUDA(cudaMalloc(&c->sym_c1f, sizeof(float) * rows));
    CPM_CUDA(cudaMemcpy(c->sym_w32, w32.data(), sizeof(float4) * rows, cudaMemcpyHostToDevice));
    CPM_CUDA(cudaMemcpy(c->sym_c1f, c1f.data(), sizeof(float) * rows, cudaMemcpyHostToDevice));
  }
  CPM_CUDA(cudaDeviceSynchronize());
  CPM_CUDA(cudaFuncSetAttribute(k_sapply_sym, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sym_smem(npad)));
  CPM_CUDA(cudaFuncSetAttribute(k_sapply_sym_tma, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sym_tma_smem()));
  c->sym_nt = nt;
  c->sym_ok = true;
  return CPM_OK;
}

// Whether the packed S-apply forms the projection sums itself (and the finish pass is left out):
// with few tiles per CTA the finish pass's fixed latency outweighs the sums' integer work in every
// tile epilogue (measured on GB300: the paper-scale cell, about two tiles per CTA, gains about
// 3 us per step; the 40,320-site doubled cell, about 83 tiles per CTA and block, loses about 10).
bool cpm_internal_sym_fuse(const cpm_ctx* c) {
  return c->sym_ok && c->sym_w32 != nullptr && sy_tiles(c->sym_nt) <= (long long)SY_FUSE_TILES_PER_CTA * c->n_sm;
}

// One S-apply of block blk (0, or 1 for the S- mirror block) from the packed tiles.  With
// fuse_sums the kernel also accumulates the projection sums and leaves q_raw - dpsi S v in qpart
// for the projection kernel to finish; otherwise k_sapply_finish writes q_raw to qout.
int cpm_internal_sapply_sym(cpm_ctx* c, int blk, const float* xh, const float* xl, const double* b,
                            const double* dpsi, const double* Sv, const double* W, const double* c1, double* qout,
                            cudaStream_t st, bool fuse_sums) {
  const int n = c->mirror ? c->nh : c->ne;
  const int nt = c->sym_nt, npad = nt * SY_T;
  const float* Sp = c->sym_S + (size_t)blk * sy_tiles(nt) * SY_T * SY_T;
  double* qpart = c->qpart + (size_t)blk * n;
  const SymSums fs = fuse_sums ? SymSums{c->sym_w32 + (size_t)blk * n, c->sym_c1f + (size_t)blk * n, c->scal}
                               : SymSums{nullptr, nullptr, nullptr};
  if (c->sapply_variant == CPM_SAPPLY_SYM_TMA)
    CPM_CUDA(launch_pdl(k_sapply_sym_tma, c->n_sm, SY_THREADS, sym_tma_smem(), st, Sp, nt, n, xh, xl, qpart,
                        c->wait_test ? 1 : 0, c->status, fs));
  else
    CPM_CUDA(launch_pdl(k_sapply_sym, c->n_sm, SY_THREADS, sym_smem(npad), st, Sp, nt, n, xh, xl, qpart, npad, fs));
  ++c->launches;
  CPM_LAUNCH();
  if (fuse_sums) return CPM_OK;
  CPM_CUDA(launch_pdl(k_sapply_finish, (n + FIN_THREADS - 1) / FIN_THREADS, FIN_THREADS, 0, st, n, qpart, b, dpsi, Sv, W, c1, qout, c->scal));
  ++c->launches;
  CPM_LAUNCH();
  return CPM_OK;
}
