// S-apply from symmetric packed storage (mixed precision, one replica): q = S (b + dpsi v) with
// S = O A^-1 (Eqs. 8-9) or, per mirror block of the doubled cell, the block's projected inverse
// (Eqs. 13-15).
//
// S (or each mirror block S+-) is symmetric, so only its upper triangle of 128 x 128 tiles is kept:
// tile (I, J), I <= J, at packed index I nt - I (I - 1) / 2 + (J - I), each tile row-major
// (diagonal tiles in full).  One read of an off-diagonal tile serves both S_IJ x_J (rows of block I)
// and S_IJ^T x_I (rows of block J), so the HBM bytes per step are about half of the full matrix.
// Partial sums have one writer each: part[J][rows of I] holds tile (I, J)'s row products and
// part[I][rows of J] its transposed products, so for every row block R the slots 0..nt-1 are
// written exactly once per call (J >= R from its row tiles, I < R from its column tiles).  The
// finish kernel sums the nt slots of each row (compensated float32), adds dpsi S v and the
// projection sums as the other S-apply variants do.
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
                                                             const float* __restrict__ xl, float* __restrict__ part,
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
      part[(size_t)J * npad + I * SY_T + tid] = (float)a.value();
      if (I != J) {
        Acc<float> b;
        for (int w = 0; w < SY_THREADS / 32; ++w) b.add(C[w * SY_T + tid]);
        part[(size_t)I * npad + J * SY_T + tid] = (float)b.value();
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

// q_raw = sum of the nt slots + dpsi S v, with the projection sums (one replica).
// Row totals from the per-tile-row partial slots: 32 rows per block, eight threads per row each
// summing every eighth slot (compensated float32), combined in shared memory; then the row's q_raw
// and its contributions to the projection sums.
constexpr int SF_ROWS = 32, SF_SPLIT = 8;
__global__ void __launch_bounds__(SF_ROWS * SF_SPLIT) k_sym_finish(int rows, int nt, int npad,
                                                                  const float* __restrict__ part,
                                                                  const double* __restrict__ b,
                                                                  const double* __restrict__ dpsi,
                                                                  const double* __restrict__ Sv,
                                                                  const double* __restrict__ W,
                                                                  const double* __restrict__ c1,
                                                                  double* __restrict__ qout, double* __restrict__ scal) {
  pdl_enter();
  __shared__ float ps[SF_SPLIT][SF_ROWS][2];
  const int r = threadIdx.x & (SF_ROWS - 1), k = threadIdx.x / SF_ROWS;
  const int i = blockIdx.x * SF_ROWS + r;
  Acc<float> a;
  if (i < rows) {
    // eight independent loads in flight per round: the slots sit in different DRAM pages
    for (int s = k; s < nt; s += 8 * SF_SPLIT) {
      float v[8];
#pragma unroll
      for (int u = 0; u < 8; ++u) {
        const int su = s + u * SF_SPLIT;
        v[u] = su < nt ? part[(size_t)su * npad + i] : 0.f;
      }
#pragma unroll
      for (int u = 0; u < 8; ++u) a.add(v[u]);
    }
  }
  ps[k][r][0] = a.s;
  ps[k][r][1] = a.c;
  __syncthreads();
  double red[4] = {0, 0, 0, 0};
  if (k == 0 && i < rows) {
    Acc<float> t;
    for (int j = 0; j < SF_SPLIT; ++j) {
      t.add(ps[j][r][0]);
      t.c += ps[j][r][1];
    }
    const double qr = t.value() + dpsi[0] * Sv[i];
    qout[i] = qr;
    const double bi = b[i];
    red[0] = qr;
    red[1] = qr * c1[i];
    red[2] = W[2 * i] * bi;
    red[3] = W[2 * i + 1] * bi;
  }
#pragma unroll
  for (int q = 0; q < 4; ++q) red[q] = warp_sum(red[q]);
  double* const dst[4] = {scal + S_CQ0, scal + S_CQ1, scal + S_WB0, scal + S_WB1};
  block_atomic_add<4>(red, dst);
}

static size_t sym_smem(int npad) { return sizeof(float) * (2 * (size_t)npad + SY_T * 33 + 8 * SY_T); }

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
  const int blocks = c->mirror ? 2 : 1;
  const long long tiles = sy_tiles(nt);
  CPM_CUDA(cudaMalloc(&c->sym_S, sizeof(float) * (size_t)blocks * tiles * SY_T * SY_T));
  CPM_CUDA(cudaMalloc(&c->sym_part, sizeof(float) * (size_t)nt * npad));
  for (int blk = 0; blk < blocks; ++blk) {
    const double* S = c->S64 + (size_t)blk * n * c->ld64;
    k_pack_sym<<<dim3(nt, nt), 256>>>(S, n, c->ld64, nt, c->sym_S + (size_t)blk * tiles * SY_T * SY_T);
    CPM_LAUNCH();
  }
  CPM_CUDA(cudaDeviceSynchronize());
  CPM_CUDA(cudaFuncSetAttribute(k_sapply_sym, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sym_smem(npad)));
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
  CPM_CUDA(launch_pdl(k_sapply_sym, c->n_sm, SY_THREADS, sym_smem(npad), st, Sp, nt, n, xh, xl, c->sym_part, npad));
  ++c->launches;
  CPM_LAUNCH();
  CPM_CUDA(launch_pdl(k_sym_finish, (n + SF_ROWS - 1) / SF_ROWS, SF_ROWS * SF_SPLIT, 0, st, n, nt, npad, c->sym_part, b,
                      dpsi, Sv, W, c1, qout, c->scal));
  ++c->launches;
  CPM_LAUNCH();
  return CPM_OK;
}
