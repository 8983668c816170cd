// SPME charge assignment and force interpolation through shared-memory bricks moved by the
// Tensor Memory Accelerator (float32 mesh, mixed precision): the reciprocal-space part of the Ewald
// sums behind Eq. 3 (Sec. II.B), for b and for the forces.
//
// The mesh gets a halo-padded twin: padded index p = g + P per axis, where g in [-P, K) is the
// unwrapped mesh index of a B-spline stencil point, so no stencil of a site ever wraps.  A block
// handles one super-cell (S0 x S1 x S2 real-space cells of the cell-sorted sites):
//   spread: the block accumulates its sites' B-spline charges into a shared-memory brick covering
//           the super-cell's stencils, then adds the brick into the padded mesh with one TMA
//           reduction (cp.reduce.async.bulk.tensor ... .add); k_mesh_fold then folds the halo
//           onto the periodic K1 x K2 x K3 mesh that the transforms use;
//   gather: after the convolution k_mesh_halo writes the periodic potential into the padded mesh,
//           and the block loads its brick with one TMA tensor load (mbarrier completion, bounded
//           wait) and interpolates forces for its sites from shared memory.
// Every box starts at a non-negative padded coordinate whose innermost (z) component is a multiple
// of 4 floats (16 bytes), and no box reaches past the padded extents, so no TMA access is out of
// range by construction.
#include "cpm_internal.cuh"

#include <cudaTypedefs.h>

#include <algorithm>
#include <vector>

namespace cpm {

constexpr int BR_THREADS = 256;
constexpr int BR_WARPS = BR_THREADS / 32;
constexpr long long BR_WAIT_LIMIT = 1LL << 22;     // mbarrier polls before a load is declared lost

struct BrickGeom {
  int S[3];          // real-space cells per super-cell per axis
  int ns[3];         // super-cells per axis
  int nc[3];         // real-space cells per axis
  int B[3];          // box extent per axis (x, y, z), mesh points
  int Kp[3];         // padded mesh extent per axis (x, y, z)
  int K[3];
  int off;           // padded index = mesh index + off (= P)
  long long Mp_s;    // per-replica stride of the padded mesh (floats)
};

__device__ __forceinline__ uint32_t br_smem(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }

// Mesh-index range of the stencil bases of cells [c0, c1) along one axis, and the padded start of
// the box (z: rounded down to a multiple of 4).
__host__ __device__ __forceinline__ int br_start(int c0, int K, int nc, int d) {
  const int lo = (c0 * K) / nc;          // floor(c0 K / nc): lowest base index (before the -1 safety)
  return d == 2 ? (lo & ~3) : lo;        // padded start = (lo - P - 1 + 1) + P ... = lo (off = P)
}

// Adds the B-spline charges of every site of one source set in the block's super-cell.
template <typename V4>
__device__ __forceinline__ void brick_spread_set(float* brick, const BrickGeom& bg, const SpmeGeom& sg,
                                                 const V4* __restrict__ loc, const int* __restrict__ start,
                                                 const int* __restrict__ sorted, const float* __restrict__ q,
                                                 const int* __restrict__ splI, const float* __restrict__ splF,
                                                 const int* cmin, const int* cmax, const int* bs,
                                                 float (*sw)[3][PMAX], float (*sdw)[3][PMAX], int (*si0)[3],
                                                 int* status) {
  const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5;
  const int P = sg.P;
  for (int cx = cmin[0]; cx < cmax[0]; ++cx)
    for (int cy = cmin[1]; cy < cmax[1]; ++cy)
      for (int cz = cmin[2]; cz < cmax[2]; ++cz) {
        const int flat = (cx * bg.nc[1] + cy) * bg.nc[2] + cz;
        const int a = start[flat], e = start[flat + 1];
        for (int k = a + wib; k < e; k += BR_WARPS) {
          V4 p = loc[k];
          const float qk = q ? q[sorted[k]] : p.w;
          site_weights<float>(p, make_int4(cx, cy, cz, flat), sg, splI, splF, lane, sw[wib], sdw[wib], si0[wib]);
          for (int task = lane; task < P * P; task += 32) {
            const int ty = task / P, tz = task - ty * P;
            const int ly = si0[wib][1] - ty + bg.off - bs[1];
            const int lz = si0[wib][2] - tz + bg.off - bs[2];
            const float wyz = qk * sw[wib][1][ty] * sw[wib][2][tz];
            for (int tx = 0; tx < P; ++tx) {
              const int lx = si0[wib][0] - tx + bg.off - bs[0];
              if ((unsigned)lx < (unsigned)bg.B[0] && (unsigned)ly < (unsigned)bg.B[1] &&
                  (unsigned)lz < (unsigned)bg.B[2])
                atomicAdd(&brick[((size_t)lx * bg.B[1] + ly) * bg.B[2] + lz], sw[wib][0][tx] * wyz);
              else
                latch_error(status, DE_DOMAIN);
            }
          }
          __syncwarp();
        }
      }
}

// One block per (super-cell, replica): spread set 0 (and set 1 when loc1 != nullptr) into a
// shared-memory brick, then one TMA reduction of the brick into the padded mesh.
template <typename V4>
__global__ void __launch_bounds__(BR_THREADS) k_spread_brick(const __grid_constant__ CUtensorMap map, BrickGeom bg,
                                                             SpmeGeom sg, const V4* __restrict__ loc0,
                                                             long long loc0_stride, const int* __restrict__ start0,
                                                             long long start0_stride, const V4* __restrict__ loc1,
                                                             const int* __restrict__ start1,
                                                             const int* __restrict__ sorted1,
                                                             const float* __restrict__ q1, int q1_stride,
                                                             const int* __restrict__ splI,
                                                             const float* __restrict__ splF, int* status) {
  extern __shared__ __align__(128) float br_dyn[];
  __shared__ float sw[BR_WARPS][3][PMAX], sdw[BR_WARPS][3][PMAX];
  __shared__ int si0[BR_WARPS][3];
  const int rep = blockIdx.y;
  const int scell = blockIdx.x;
  const int sz = scell % bg.ns[2], sy = (scell / bg.ns[2]) % bg.ns[1], sx = scell / (bg.ns[2] * bg.ns[1]);
  const int sc[3] = {sx, sy, sz};
  int cmin[3], cmax[3], bs[3];
  for (int d = 0; d < 3; ++d) {
    cmin[d] = sc[d] * bg.S[d];
    cmax[d] = min(bg.nc[d], cmin[d] + bg.S[d]);
    bs[d] = br_start(cmin[d], bg.K[d], bg.nc[d], d);
  }
  // skip empty super-cells (uniform over the block)
  const int* st0 = start0 + rep * start0_stride;
  int nsite = 0;
  for (int cx = cmin[0]; cx < cmax[0]; ++cx)
    for (int cy = cmin[1]; cy < cmax[1]; ++cy) {
      const int f0 = (cx * bg.nc[1] + cy) * bg.nc[2];
      nsite += st0[f0 + cmax[2]] - st0[f0 + cmin[2]];
      if (loc1) nsite += start1[f0 + cmax[2]] - start1[f0 + cmin[2]];
    }
  if (nsite == 0) return;
  const int nb = bg.B[0] * bg.B[1] * bg.B[2];
  for (int k = threadIdx.x; k < nb; k += BR_THREADS) br_dyn[k] = 0.f;
  __syncthreads();
  brick_spread_set<V4>(br_dyn, bg, sg, loc0 + rep * loc0_stride, st0, nullptr, nullptr, splI, splF, cmin, cmax, bs,
                       sw, sdw, si0, status);
  if (loc1)
    brick_spread_set<V4>(br_dyn, bg, sg, loc1, start1, sorted1, q1 + (size_t)rep * q1_stride, splI, splF, cmin,
                         cmax, bs, sw, sdw, si0, status);
  __syncthreads();
  if (threadIdx.x == 0) {
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    asm volatile(
        "cp.reduce.async.bulk.tensor.4d.global.shared::cta.add.tile.bulk_group [%0, {%1, %2, %3, %4}], [%5];" ::"l"(
            reinterpret_cast<uint64_t>(&map)),
        "r"(bs[2]), "r"(bs[1]), "r"(bs[0]), "r"(rep), "r"(br_smem(br_dyn))
        : "memory");
    asm volatile("cp.async.bulk.commit_group;" ::: "memory");
    asm volatile("cp.async.bulk.wait_group.read 0;" ::: "memory");
  }
}

// periodic mesh <- padded mesh folded: m[g] = sum over p = g + off (mod K) inside the padded extents
// (per axis the padded images of g are listed first: one for interior points, two near the faces).
__global__ void __launch_bounds__(256) k_mesh_fold(const float* __restrict__ pad, float* __restrict__ mesh,
                                                   BrickGeom bg, long long Mr_s) {
  const int rep = blockIdx.y;
  const long long M = (long long)bg.K[0] * bg.K[1] * bg.K[2];
  const float* pr = pad + (size_t)rep * bg.Mp_s;
  float* mr = mesh + (size_t)rep * Mr_s;
  for (long long g = blockIdx.x * (long long)blockDim.x + threadIdx.x; g < M; g += (long long)gridDim.x * blockDim.x) {
    const int gi[3] = {(int)(g / ((long long)bg.K[2] * bg.K[1])), (int)((g / bg.K[2]) % bg.K[1]), (int)(g % bg.K[2])};
    int pv[3][3], np[3];
#pragma unroll
    for (int d = 0; d < 3; ++d) {
      np[d] = 0;
      for (int p = (gi[d] + bg.off) % bg.K[d]; p < bg.Kp[d]; p += bg.K[d])
        if (np[d] < 3) pv[d][np[d]++] = p;
    }
    float s = 0.f;
    for (int a = 0; a < np[0]; ++a)
      for (int b = 0; b < np[1]; ++b) {
        const float* row = pr + ((size_t)pv[0][a] * bg.Kp[1] + pv[1][b]) * bg.Kp[2];
        for (int e = 0; e < np[2]; ++e) s += row[pv[2][e]];
      }
    mr[g] = s;
  }
}

// padded mesh <- periodic potential: pad[p] = phi[(p - off) mod K] per axis.
__global__ void __launch_bounds__(256) k_mesh_halo(const float* __restrict__ phi, float* __restrict__ pad,
                                                   BrickGeom bg, long long Mr_s) {
  const int rep = blockIdx.y;
  const long long M = (long long)bg.Kp[0] * bg.Kp[1] * bg.Kp[2];
  const float* src = phi + (size_t)rep * Mr_s;
  float* dst = pad + (size_t)rep * bg.Mp_s;
  for (long long p = blockIdx.x * (long long)blockDim.x + threadIdx.x; p < M; p += (long long)gridDim.x * blockDim.x) {
    const int pz = (int)(p % bg.Kp[2]), py = (int)((p / bg.Kp[2]) % bg.Kp[1]),
              px = (int)(p / ((long long)bg.Kp[2] * bg.Kp[1]));
    const int gx = wrap_index(px - bg.off, bg.K[0]), gy = wrap_index(py - bg.off, bg.K[1]),
              gz = wrap_index(pz - bg.off, bg.K[2]);
    dst[p] = src[((size_t)gx * bg.K[1] + gy) * bg.K[2] + gz];
  }
}

// One block per (super-cell, replica): TMA load of the potential brick, then for every electrolyte
// site of the super-cell F = -Q grad(phi_mesh) + Q E_z z-hat + the real-space force f_pair, written at
// the site's input index (same output as k_gather_f_elyt).
template <typename V4>
__global__ void __launch_bounds__(BR_THREADS) k_gather_f_brick(const __grid_constant__ CUtensorMap map, BrickGeom bg,
                                                               SpmeGeom sg, const int* __restrict__ off, int cap,
                                                               const V4* __restrict__ loc, const int* __restrict__ start,
                                                               const int* __restrict__ sorted,
                                                               const int* __restrict__ splI,
                                                               const float* __restrict__ splF,
                                                               const double* __restrict__ dpsi, double ff_over_lz,
                                                               double slab_coef, const double* __restrict__ scal,
                                                               const double* __restrict__ f_pair,
                                                               double* __restrict__ F, int short_wait, int* status) {
  extern __shared__ __align__(128) float br_dyn[];
  __shared__ float sw[BR_WARPS][3][PMAX], sdw[BR_WARPS][3][PMAX];
  __shared__ int si0[BR_WARPS][3];
  __shared__ __align__(8) uint64_t mbar;
  __shared__ int ok;
  const int rep = blockIdx.y;
  const int scell = blockIdx.x;
  const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5;
  const int sz = scell % bg.ns[2], sy = (scell / bg.ns[2]) % bg.ns[1], sx = scell / (bg.ns[2] * bg.ns[1]);
  const int sc[3] = {sx, sy, sz};
  int cmin[3], cmax[3], bs[3];
  for (int d = 0; d < 3; ++d) {
    cmin[d] = sc[d] * bg.S[d];
    cmax[d] = min(bg.nc[d], cmin[d] + bg.S[d]);
    bs[d] = br_start(cmin[d], bg.K[d], bg.nc[d], d);
  }
  const int* st = start + rep * (long long)(bg.nc[0] * bg.nc[1] * bg.nc[2] + 1);
  int nsite = 0;
  for (int cx = cmin[0]; cx < cmax[0]; ++cx)
    for (int cy = cmin[1]; cy < cmax[1]; ++cy) {
      const int f0 = (cx * bg.nc[1] + cy) * bg.nc[2];
      nsite += st[f0 + cmax[2]] - st[f0 + cmin[2]];
    }
  if (nsite == 0) return;
  const uint32_t bytes = (uint32_t)(sizeof(float) * bg.B[0] * bg.B[1] * bg.B[2]);
  if (threadIdx.x == 0) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(br_smem(&mbar)), "r"(1) : "memory");
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(br_smem(&mbar)), "r"(bytes) : "memory");
    asm volatile(
        "cp.async.bulk.tensor.4d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3, %4, %5}], "
        "[%6];" ::"r"(br_smem(br_dyn)),
        "l"(reinterpret_cast<uint64_t>(&map)), "r"(bs[2]), "r"(bs[1]), "r"(bs[0]), "r"(rep), "r"(br_smem(&mbar))
        : "memory");
  }
  // bounded wait for the brick (phase 0); short_wait (cpm_set_wait_test) makes it give up without
  // polling
  if (threadIdx.x == 0) {
    uint32_t done = 0;
    const long long first_limit = short_wait ? 0 : BR_WAIT_LIMIT;
    for (long long it = 0; it < first_limit && !done; ++it) {
      asm volatile("{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}"
                   : "=r"(done)
                   : "r"(br_smem(&mbar)), "r"(0)
                   : "memory");
      if (!done) __nanosleep(32);
    }
    ok = (int)done;
    if (!done) {
      latch_error(status, DE_TIMEOUT);
      // a second bounded wait for the copy still in flight into this block's shared memory
      for (long long it = 0; it < BR_WAIT_LIMIT && !done; ++it) {
        asm volatile("{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}"
                     : "=r"(done)
                     : "r"(br_smem(&mbar)), "r"(0)
                     : "memory");
        if (!done) __nanosleep(32);
      }
    }
  }
  __syncthreads();
  if (!ok) return;       // the brick is not used after a timed-out load
  const int P = sg.P;
  const int o = off[rep];
  const V4* lr = loc + (size_t)rep * cap;
  const int* so = sorted + (size_t)rep * cap;
  const double mz = scal[rep * NSCAL + S_QZ_ELYT] + scal[rep * NSCAL + S_QZ_ELEC];
  const double ezf = -dpsi[rep] * ff_over_lz - slab_coef * mz;
  for (int cx = cmin[0]; cx < cmax[0]; ++cx)
    for (int cy = cmin[1]; cy < cmax[1]; ++cy)
      for (int cz = cmin[2]; cz < cmax[2]; ++cz) {
        const int flat = (cx * bg.nc[1] + cy) * bg.nc[2] + cz;
        for (int k = st[flat] + wib; k < st[flat + 1]; k += BR_WARPS) {
          const V4 p = lr[k];
          site_weights<float>(p, make_int4(cx, cy, cz, flat), sg, splI, splF, lane, sw[wib], sdw[wib], si0[wib]);
          float gx = 0.f, gy = 0.f, gz = 0.f;
          for (int task = lane; task < P * P; task += 32) {
            const int ty = task / P, tz = task - ty * P;
            const int ly = si0[wib][1] - ty + bg.off - bs[1];
            const int lz = si0[wib][2] - tz + bg.off - bs[2];
            float a = 0.f, ad = 0.f;
            for (int tx = 0; tx < P; ++tx) {
              const int lx = si0[wib][0] - tx + bg.off - bs[0];
              float ph = 0.f;
              if ((unsigned)lx < (unsigned)bg.B[0] && (unsigned)ly < (unsigned)bg.B[1] &&
                  (unsigned)lz < (unsigned)bg.B[2])
                ph = br_dyn[((size_t)lx * bg.B[1] + ly) * bg.B[2] + lz];
              else
                latch_error(status, DE_DOMAIN);
              a += sw[wib][0][tx] * ph;
              ad += sdw[wib][0][tx] * ph;
            }
            const float wy = sw[wib][1][ty], wz = sw[wib][2][tz];
            gx += ad * wy * wz;
            gy += a * sdw[wib][1][ty] * wz;
            gz += a * wy * sdw[wib][2][tz];
          }
          gx = warp_sum(gx);
          gy = warp_sum(gy);
          gz = warp_sum(gz);
          if (lane == 0) {
            const double q = (double)p.w;
            const int i = so[k];
            const size_t gi = 3 * (size_t)(o + i);
            const double* fp = f_pair + 3 * ((size_t)rep * cap + i);
            F[gi + 0] = -q * (double)gx * sg.kl[0] + fp[0];
            F[gi + 1] = -q * (double)gy * sg.kl[1] + fp[1];
            F[gi + 2] = -q * (double)gz * sg.kl[2] + q * ezf + fp[2];
          }
          __syncwarp();
        }
      }
}

static BrickGeom brick_geom(const cpm_ctx* c) {
  BrickGeom bg;
  for (int d = 0; d < 3; ++d) {
    bg.S[d] = c->br_S[d];
    bg.nc[d] = c->nc[d];
    bg.ns[d] = (c->nc[d] + bg.S[d] - 1) / bg.S[d];
    bg.B[d] = c->br_B[d];
    bg.Kp[d] = c->br_Kp[d];
    bg.K[d] = c->K[d];
  }
  bg.off = c->P;
  bg.Mp_s = c->br_Mp_s;
  return bg;
}

}  // namespace cpm

using namespace cpm;

// Brick geometry, padded mesh and its tensor map (mixed precision).  Leaves c->brick_ok false when
// a box would not fit the shared-memory budget or the tensor map cannot be encoded.
int cpm_internal_brick_setup(cpm_ctx* c) {
  c->brick_ok = false;
  if (!c->mixed) return CPM_OK;
  const int P = c->P;
  int Kp[3], B[3];
  for (int d = 0; d < 3; ++d) {
    const int nc = c->nc[d], K = c->K[d];
    c->br_S[d] = nc >= 4 ? 2 : 1;
    const int S = c->br_S[d];
    const int ns = (nc + S - 1) / S;
    int need = 0, ext = 0;
    for (int s = 0; s < ns; ++s) {
      const int c0 = s * S, c1 = std::min(nc, c0 + S);
      const int start = br_start(c0, K, nc, d);
      const int hi = (c1 * K + nc - 1) / nc;                 // ceil(c1 K / nc): highest base + 1 (safety incl.)
      const int last = hi + P;                              // highest padded index needed: (hi) - 0 + off
      need = std::max(need, last - start + 1);
      ext = std::max(ext, start + 0);
    }
    if (d == 2) need = (need + 3) & ~3;
    B[d] = need;
    int kp = 0;
    for (int s = 0; s < ns; ++s) kp = std::max(kp, br_start(s * S, K, nc, d) + B[d]);
    if (d == 2) kp = (kp + 3) & ~3;
    Kp[d] = kp;
    (void)ext;
  }
  const size_t box_bytes = sizeof(float) * (size_t)B[0] * B[1] * B[2];
  if (box_bytes > 96 * 1024 || B[0] > 256 || B[1] > 256 || B[2] > 256) return CPM_OK;
  for (int d = 0; d < 3; ++d) {
    c->br_B[d] = B[d];
    c->br_Kp[d] = Kp[d];
  }
  const long long Mp = (long long)Kp[0] * Kp[1] * Kp[2];
  c->br_Mp_s = (Mp + 63) & ~63LL;
  const int R = c->p.max_replicas;
  CPM_CUDA(cudaMalloc(&c->br_pad, sizeof(float) * (size_t)R * c->br_Mp_s));
  CPM_CUDA(cudaMemset(c->br_pad, 0, sizeof(float) * (size_t)R * c->br_Mp_s));
  void* fn = nullptr;
  cudaDriverEntryPointQueryResult qr;
  if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &fn, 12000, cudaEnableDefault, &qr) != cudaSuccess ||
      qr != cudaDriverEntryPointSuccess || !fn) {
    set_error("cuTensorMapEncodeTiled is not available from the driver");
    return CPM_OK;
  }
  auto encode = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(fn);
  const cuuint64_t dims[4] = {(cuuint64_t)Kp[2], (cuuint64_t)Kp[1], (cuuint64_t)Kp[0], (cuuint64_t)R};
  const cuuint64_t strides[3] = {sizeof(float) * (cuuint64_t)Kp[2], sizeof(float) * (cuuint64_t)Kp[2] * Kp[1],
                                 sizeof(float) * (cuuint64_t)c->br_Mp_s};
  const cuuint32_t box[4] = {(cuuint32_t)B[2], (cuuint32_t)B[1], (cuuint32_t)B[0], 1};
  const cuuint32_t estr[4] = {1, 1, 1, 1};
  const CUresult r = encode(&c->br_map, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 4, c->br_pad, dims, strides, box, estr,
                            CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE,
                            CU_TENSOR_MAP_L2_PROMOTION_L2_128B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  if (r != CUDA_SUCCESS) {
    set_error("cuTensorMapEncodeTiled failed (%d) for the padded mesh", (int)r);
    return CPM_OK;
  }
  CPM_CUDA(cudaFuncSetAttribute(k_spread_brick<float4>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)box_bytes));
  CPM_CUDA(cudaFuncSetAttribute(k_gather_f_brick<float4>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                (int)box_bytes));
  c->brick_ok = true;
  return CPM_OK;
}

static int nsuper(const cpm_ctx* c) {
  int n = 1;
  for (int d = 0; d < 3; ++d) n *= (c->nc[d] + c->br_S[d] - 1) / c->br_S[d];
  return n;
}

// Electrolyte charges (and, with the electrode charges qT != nullptr, the electrode charges) onto
// the periodic mesh c->mesh_r through the padded mesh: clear, brick spread + TMA reductions, fold.
int cpm_internal_spread_brick(cpm_ctx* c, int nrep, const void* l_loc, const float* qT, cudaStream_t st) {
  const BrickGeom bg = brick_geom(c);
  SpmeGeom sg = cpm_internal_spme_geom(c);
  const size_t box_bytes = sizeof(float) * (size_t)bg.B[0] * bg.B[1] * bg.B[2];
  CPM_CUDA(cudaMemsetAsync(c->br_pad, 0, sizeof(float) * (size_t)nrep * c->br_Mp_s, st));
  const int cap = c->p.max_elyt;
  k_spread_brick<float4><<<dim3(nsuper(c), nrep), BR_THREADS, box_bytes, st>>>(
      c->br_map, bg, sg, (const float4*)l_loc, (long long)cap, c->l_start, (long long)c->ncell + 1,
      qT ? c->e_loc32 : nullptr, c->e_start, c->e_sorted, qT, c->ne, c->spl_I, c->spl_F32, c->status);
  ++c->launches;
  CPM_LAUNCH();
  const long long M = (long long)c->K[0] * c->K[1] * c->K[2];
  const int blocks = (int)std::min<long long>((M + 255) / 256, 152 * 8);
  k_mesh_fold<<<dim3(blocks, nrep), 256, 0, st>>>(c->br_pad, (float*)c->mesh_r, bg, c->Mr_s);
  ++c->launches;
  CPM_LAUNCH();
  return CPM_OK;
}

// Forces on the electrolyte from the potential c->mesh_phi: halo fill of the padded mesh, then the
// brick gather (TMA loads).  Same output as the per-site gather.
int cpm_internal_gather_f_brick(cpm_ctx* c, int nrep, const int* off, const void* l_loc, const double* dpsi,
                                double ff_over_lz, double slab_coef, double* F, cudaStream_t st) {
  const BrickGeom bg = brick_geom(c);
  SpmeGeom sg = cpm_internal_spme_geom(c);
  const size_t box_bytes = sizeof(float) * (size_t)bg.B[0] * bg.B[1] * bg.B[2];
  const long long Mp = (long long)bg.Kp[0] * bg.Kp[1] * bg.Kp[2];
  const int blocks = (int)std::min<long long>((Mp + 255) / 256, 152 * 8);
  k_mesh_halo<<<dim3(blocks, nrep), 256, 0, st>>>((const float*)c->mesh_phi, c->br_pad, bg, c->Mr_s);
  ++c->launches;
  CPM_LAUNCH();
  k_gather_f_brick<float4><<<dim3(nsuper(c), nrep), BR_THREADS, box_bytes, st>>>(
      c->br_map, bg, sg, off, c->p.max_elyt, (const float4*)l_loc, c->l_start, c->l_sorted, c->spl_I, c->spl_F32,
      dpsi, ff_over_lz, slab_coef, c->scal, c->f_pair, F, c->wait_test ? 1 : 0, c->status);
  ++c->launches;
  CPM_LAUNCH();
  return CPM_OK;
}
