// Internal definitions shared by the CPM library translation units: the context layout, error
// plumbing, and small device helpers (cardinal B-splines, warp reductions, cell geometry).
#pragma once

#include <cuda.h>
#include <cuda_runtime.h>
#include <cufft.h>
#include <cublas_v2.h>
#include <cusolverDn.h>

#include <cmath>
#include <cstdint>
#include <cstdio>
#include <string>
#include <vector>

#include "../../include/cpm.h"

namespace cpm {

constexpr double KE = 14.3996454784;        // e^2 / (4 pi eps0), eV A
constexpr double PI = 3.14159265358979323846;
constexpr int PMAX = 8;                     // largest supported B-spline order
constexpr int NSCAL = 18;                   // per-replica float64 scalar slots
constexpr int kMaxStencil = 512;            // neighbour-cell stencil entries of the pair kernel
constexpr int kEeTabMax = 4096;             // distinct G vectors of the compressed electrode pair list
                                            // (float4, in 64 KB of shared memory), zero entry included

// Per-replica scalar slots (float64 accumulators, zeroed at the start of every call).
enum Slot {
  S_QZ_ELYT = 0,   // sum_j Q_j Z_j
  S_QQ_ELYT = 1,   // sum_j Q_j^2
  S_QZ_ELEC = 2,   // sum_i q_i z_i
  S_QV_ELEC = 3,   // sum_i q_i v_i
  S_QQ_ELEC = 4,   // sum_i q_i^2
  S_E_LL = 5,      // sum_j Q_j phi^pp_j            (real space, no KE)
  S_E_LE = 6,      // sum_j Q_j phi^gp_j            (real space, no KE)
  S_E_EE = 7,      // sum_i q_i phi^gg_i            (real space, no KE)
  S_E_RECIP = 8,   // 1/2 sum_m G |rho^(m)|^2       (eV)
  S_CQ0 = 9,       // e^T q_raw
  S_CQ1 = 10,      // e_1^T q_raw
  S_WB0 = 11,      // (A^-1 e)^T b
  S_WB1 = 12,      // (A^-1 e_1)^T b
  S_E_RECIP_L = 13,// 1/2 sum_m G |rho_elyt^(m)|^2 (eV), electrolyte charges alone
  S_QB = 14,       // q^T b (after the projection)
  S_QPLUS = 15,    // sum of q over side +1 sites
  S_E_LJ = 16      // Lennard-Jones energy of the electrolyte (eV), when an MD run enables it
};

// Lennard-Jones interactions of an MD run (cpm_md_run), evaluated by the step's electrolyte-target
// pair kernel while the run holds the context (ctx->lj set for its duration).
constexpr int kLjMaxTypes = 8;
struct LjSetup {
  const int* type = nullptr;    // [offsets[n_rep]] LJ type per electrolyte site (replica-major)
  int elec_type = -1;           // type of every electrode site, -1: no electrode interaction
  double cut = 0.0;             // force-shifted cutoff (A), <= rcut
  double sig_half[kLjMaxTypes] = {};   // sigma / 2 (Lorentz-Berthelot: sigma_ab = half_a + half_b)
  double sqrt_eps[kLjMaxTypes] = {};   // sqrt(eps) (eps_ab = sqrt_eps_a sqrt_eps_b)
};
constexpr int NENERGY = 4;                  // per-replica energy outputs: U, H, dH/d(dpsi), Q_+

// Status bits latched by kernels (first error wins).
enum DevErr { DE_NONFINITE = 1, DE_DOMAIN = 2, DE_TIMEOUT = 4, DE_CAPACITY = 8 };

void set_error(const char* fmt, ...);

}  // namespace cpm

struct cpm_ctx {
  cpm_params p;
  int dev = 0;
  int ne = 0, ncons = 1;
  bool mixed = false;
  double ebox[3] = {0, 0, 0};   // Ewald box (slab: padded z)
  double V = 0;                 // Ewald box volume
  double Lz = 0;                // physical cell length in z (finite-field ramp, field term)
  // real-space cell grid (edge >= rcut/2 per axis)
  int nc[3] = {1, 1, 1};
  double edge[3] = {0, 0, 0};
  int ncell = 1;
  int sten[3] = {0, 0, 0};      // stencil half-width per axis: ceil(rcut / edge)
  // electrode data, device
  double4_32a* e_pos64 = nullptr;   // original order (x, y, z wrapped into the box, 0)
  double4_32a* e_loc64 = nullptr;   // cell-sorted, cell-local coordinates, w = 0
  float4* e_loc32 = nullptr;
  int4* e_cellc = nullptr;      // cell-sorted: cell coords (cx, cy, cz, flat)
  int* e_sorted = nullptr;      // cell-sorted -> original index
  int* e_start = nullptr;       // [ncell + 1]
  int4* e_base = nullptr;       // original order: B-spline base grid index per axis
  double* e_th64 = nullptr;     // [ne][3][PMAX] B-spline weights
  double* e_dth64 = nullptr;    // [ne][3][PMAX] derivatives (per grid unit)
  float* e_th32 = nullptr;
  float* e_dth32 = nullptr;
  double* e_z = nullptr;        // [ne] z as given
  double* e_v = nullptr;        // [ne] geometry vector v
  double* e_c1 = nullptr;       // [ne] e_1 indicator (doubled cell) or zeros
  double* e_plus = nullptr;     // [ne] 1 on side +1 sites, else 0
  // matrices.  Full form: S64/S32 [ne][ld] (ld = ld64 = ld32), W [ne][2], Sv [ne].
  // Mirror form (doubled cell, mirror-symmetric electrode): S64/S32 = [S+ ; S-], each [nh][ldh];
  // W [2][nh][2] = rows of S+ carry (w+, 0) and rows of S- (0, w-) with w+- = A+-^-1 1; Sv = [S+ v+ ; S- v-];
  // Mh[0], Mh[1] = 1 / 1^T w+-; WTv = (w+^T v+, w-^T v-).
  int ld64 = 0, ld32 = 0;
  int ldb = 0;                  // row stride of b_tmp (ne rounded up to 4)
  int ldx = 0;                  // length of one half (hi or lo) of a replica's b32 row
  double* S64 = nullptr;        // projected inverse, float64 master
  float* S32 = nullptr;         // float copy (mixed precision)
  double* W = nullptr;          // A^-1 C (second column zero unless doubled)
  double* Sv = nullptr;
  double Mh[4] = {0, 0, 0, 0};  // (C^T A^-1 C)^-1, host
  double WTv[2] = {0, 0};       // (A^-1 C)^T v, host
  bool mirror = false;          // mirror-block form
  int nh = 0, ldh = 0;          // sites per sub-cell and the block row stride (mirror form)
  int* m_i0 = nullptr;          // [nh] original index of block row k (a sub-cell-0 site)
  int* m_j = nullptr;           // [nh] original index of its mirror image
  std::vector<int> h_i0, h_j;   // host copies
  double* e_c1m = nullptr;      // [2 nh] zeros then ones (constraint indicator of the S-apply rows)
  double* ypm = nullptr;        // [max_rep][2 ldh] y+ = b_I0 + b_m(I0), y- = b_I0 - b_m(I0)
  double* qpm = nullptr;        // [max_rep][2 nh] q+, q- before the projection
  // S-apply variant (enum cpm_sapply_variant) and the streaming and packed variants' row partial
  // sums ([rows of S], float64, zero between calls: the finish kernel, or the projection after a
  // packed S-apply that formed the projection sums itself, clears what it consumed)
  int pair_gz = 1;               // real-space pair kernels: z cells per block (cpm_set_pair_group)
  bool wait_test = false;       // cpm_set_wait_test: the first bounded mbarrier waits give up at once
  int pair_variant = 0;         // enum cpm_pair_variant
  int sapply_variant = 0;
  double* qpart = nullptr;
  // symmetric packed S (upper-triangle 128 x 128 tiles, float32) and its per-slot partial sums
  bool sym_ok = false;
  int sym_nt = 0;
  float* sym_S = nullptr;
  // inputs of the projection sums the packed S-apply forms: W = A^-1 C as float32 pairs
  // (W0 hi, W0 lo, W1 hi, W1 lo) and the c1 indicator per row of S (or of both mirror blocks),
  // and (1^T S v, c1^T S v), which the projection multiplies by dpsi
  float4* sym_w32 = nullptr;
  float* sym_c1f = nullptr;
  double sym_sv[2] = {0.0, 0.0};
  // electrode-electrode real-space force list of the frozen electrode (mixed precision): CSR rows
  // per target (original order), entries (G_x, G_y, G_z, source index as int bits); or, when the
  // G vectors take few distinct values (a lattice electrode), the compressed form: entries
  // j | t << 16 with t indexing the table ee_tab of distinct G (last entry zero), each row padded
  // with zero entries to a multiple of 4 (ee_ptr then holds the padded row starts)
  int* ee_ptr = nullptr;
  float4* ee_g = nullptr;
  unsigned* ee_idx = nullptr;
  float4* ee_tab = nullptr;
  int ee_ntab = 0;
  int ee_lpr = 8;               // lanes per row of k_ee_forces_tab, fixed by the entry order of the build
  long long ee_nnz = 0;
  int n_sm = 0;                 // streaming multiprocessors of the device (persistent grids)
  // mesh convolution variant (enum cpm_fft_variant) and the tables of this library's own
  // float32 transform: per-axis four-step split K = n1 n2 and twiddles exp(-2 pi i t / K)
  int fft_variant = 0;
  bool fft_own_ok = false;
  float2* fft_tw = nullptr;
  int fft_n1[3] = {1, 1, 1};
  int fft_tw_off[3] = {0, 0, 0};
  // mesh charge assignment / force interpolation variant (enum cpm_mesh_variant) and the
  // halo-padded mesh of the brick variant with its TMA tensor map
  int mesh_variant = 0;
  bool brick_ok = false;
  int br_S[3] = {1, 1, 1};      // real-space cells per super-cell
  int br_B[3] = {0, 0, 0};      // box extent (x, y, z)
  int br_Kp[3] = {0, 0, 0};     // padded mesh extent (x, y, z)
  long long br_Mp_s = 0;        // per-replica stride of the padded mesh
  float* br_pad = nullptr;      // [max_rep][br_Mp_s]
  CUtensorMap br_map;           // 4-D tiled map of br_pad: (z, y, x, replica), box br_B
  cudaEvent_t ev_sorted = nullptr;   // side stream: sorted cell list complete
  cudaEvent_t ev_ee = nullptr;       // side stream: electrode pair-list field complete
  double dqdpsi = 0;
  uint64_t key = 0;             // FNV-1a 64 of the inputs that determine A (matrix images)
  // SPME
  int K[3] = {0, 0, 0};
  int P = 5;
  long long Mr = 0, Mc = 0;     // real / half-complex mesh sizes per replica
  long long Mr_s = 0, Mc_s = 0; // per-replica strides, padded to 256-byte multiples
  double* G64 = nullptr;        // [Mc] influence function incl. KE and B-spline factors (V e^-1)
  float* G32 = nullptr;
  cufftHandle plan_r2c[2] = {0, 0};   // [0] batch 1, [1] batch max_replicas
  cufftHandle plan_c2r[2] = {0, 0};
  bool have_plan[2] = {false, false};
  void* mesh_r = nullptr;       // [max_rep][Mr] real mesh (charges)
  void* mesh_c = nullptr;       // [max_rep][Mc] complex spectrum
  void* mesh_phi = nullptr;     // [max_rep][Mr] potential mesh
  // electrolyte workspaces (capacity max_replicas x max_elyt)
  int* l_cell = nullptr;        // per site flat cell index
  int* l_count = nullptr;       // [max_rep][ncell]
  int* l_start = nullptr;       // [max_rep][ncell + 1]
  int* l_sorted = nullptr;      // [max_rep][max_elyt] sorted -> original (relative to offset)
  double4_32a* l_loc64 = nullptr;   // [max_rep][max_elyt] cell-local coordinates + Q
  float4* l_loc32 = nullptr;
  void* l_tmp = nullptr;        // [max_rep][max_elyt] unsorted cell-local coordinates + Q (working precision)
  void* qT = nullptr;           // [max_rep][ne] electrode charges in the working precision
  // B-spline coordinate of each cell origin along each axis: c K_d / nc_d = spl_I + spl_F
  int* spl_I = nullptr;         // [nc0 + nc1 + nc2]
  double* spl_F64 = nullptr;
  float* spl_F32 = nullptr;
  // per-replica buffers
  double* phi_real = nullptr;   // [max_rep][ne]
  double* e_field = nullptr;    // [max_rep][ne][3] electrolyte real-space field at the electrode sites (b pass)
  double* b_tmp = nullptr;      // [max_rep][ne]
  float* b32 = nullptr;         // [max_rep][2][ldx] float32 high / low split of the S-apply input (mixed)
  float* qraw32 = nullptr;      // [max_rep][ne] tensor-core S-apply output S b (mixed, batched)
  double* scal = nullptr;       // [max_rep][NSCAL]
  int* status = nullptr;        // device status word
  // per-phase event profiler
  cudaEvent_t* prof_ev = nullptr;   // [2 * prof_cap]
  int* prof_phase = nullptr;        // [prof_cap]
  int prof_cap = 0, prof_used = 0;
  long long launches = 0;           // kernels of this library launched by per-step calls
  // side stream for work independent of the mesh chain (forked and joined with events, so a
  // captured call becomes a forked CUDA graph)
  cudaStream_t side = nullptr;
  cudaEvent_t ev_fork = nullptr, ev_join = nullptr;
  double* f_pair = nullptr;     // [max_rep][max_elyt][3] real-space electrolyte forces (original order)
  float* f_sorted32 = nullptr;  // [max_rep][max_elyt][3] the same from the third-law kernel (sorted order)
  const cpm::LjSetup* lj = nullptr;  // Lennard-Jones of a running MD loop (added into f_pair), or none
  // libraries
  cublasHandle_t cublas = nullptr;
  cusolverDnHandle_t solver = nullptr;
};

// ------------------------------------------------------------------------------------------
// error plumbing
// ------------------------------------------------------------------------------------------
#define CPM_CUDA(call)                                                                         \
  do {                                                                                         \
    cudaError_t e_ = (call);                                                                   \
    if (e_ != cudaSuccess) {                                                                   \
      cpm::set_error("%s:%d %s: %s", __FILE__, __LINE__, #call, cudaGetErrorString(e_));      \
      return (e_ == cudaErrorMemoryAllocation) ? CPM_ERR_NOMEM : CPM_ERR_CUDA;                 \
    }                                                                                          \
  } while (0)

#define CPM_LAUNCH()                                                                           \
  do {                                                                                         \
    cudaError_t e_ = cudaGetLastError();                                                       \
    if (e_ != cudaSuccess) {                                                                   \
      cpm::set_error("%s:%d kernel launch: %s", __FILE__, __LINE__, cudaGetErrorString(e_));  \
      return CPM_ERR_CUDA;                                                                     \
    }                                                                                          \
  } while (0)

#define CPM_LIB(cond, what)                                                                    \
  do {                                                                                         \
    if (!(cond)) {                                                                             \
      cpm::set_error("%s:%d %s failed", __FILE__, __LINE__, what);                             \
      return CPM_ERR_LIBRARY;                                                                  \
    }                                                                                          \
  } while (0)

#define CPM_TRY(expr)                                                                          \
  do {                                                                                         \
    int s_ = (expr);                                                                           \
    if (s_ != CPM_OK) return s_;                                                               \
  } while (0)

// ------------------------------------------------------------------------------------------
// device helpers
// ------------------------------------------------------------------------------------------
namespace cpm {

template <typename T> struct Vec4;
template <> struct Vec4<float> { using type = float4; };
template <> struct Vec4<double> { using type = double4_32a; };

__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

__device__ __forceinline__ float warp_sum(float v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

// Neumaier compensated accumulation (used for float32 running sums).
template <typename T> struct CompSum {
  T s = 0, c = 0;
  __device__ __forceinline__ void add(T x) {
    T t = s + x;
    c += (fabs(s) >= fabs(x)) ? ((s - t) + x) : ((x - t) + s);
    s = t;
  }
  __device__ __forceinline__ double value() const { return (double)s + (double)c; }
};

// Cardinal B-spline weights of order p at fractional offset f in [0, 1):
// w[t] = M_p(f + t) belongs to mesh point (floor(u) - t); dw[t] = d M_p / du there.
// Recursion M_n(x) = [x M_{n-1}(x) + (n - x) M_{n-1}(x - 1)] / (n - 1), and
// M_n'(x) = M_{n-1}(x) - M_{n-1}(x - 1) (Essmann et al., J. Chem. Phys. 103, 8577 (1995)).
// In float32 the weights are rescaled to sum to one (the partition of unity of the B-splines):
// the rounded reciprocals 1/(n - 1) of the recursion scale every weight of every site by the same
// factor, 1 + O(p 2^-24), which would bias each charge's mesh self-energy (hundreds of eV in a
// cell, cancelled by the exact Ewald self term) by the same relative amount.
template <typename T>
__device__ __forceinline__ void bspline(T f, int p, T* w, T* dw) {
#pragma unroll
  for (int t = 0; t < PMAX; ++t) { w[t] = 0; dw[t] = 0; }
  w[0] = 1;
#pragma unroll
  for (int n = 2; n <= PMAX; ++n) {
    if (n > p) break;
    if (n == p) {
#pragma unroll
      for (int t = 0; t < PMAX; ++t) {
        if (t >= n) break;
        dw[t] = w[t] - (t > 0 ? w[t - 1] : T(0));
      }
    }
    const T inv = T(1) / T(n - 1);
#pragma unroll
    for (int t = PMAX - 1; t >= 0; --t) {
      if (t >= n) continue;
      const T a = (t < n - 1) ? w[t] : T(0);
      const T b = (t > 0) ? w[t - 1] : T(0);
      w[t] = ((f + T(t)) * a + (T(n) - f - T(t)) * b) * inv;
    }
  }
  if (sizeof(T) == sizeof(float)) {
    T sum = 0;
#pragma unroll
    for (int t = 0; t < PMAX; ++t) sum += (t < p) ? w[t] : T(0);
    const T norm = T(1) / sum;
#pragma unroll
    for (int t = 0; t < PMAX; ++t) w[t] *= norm;
  }
}

__device__ __forceinline__ int wrap_index(int i, int n) {
  i %= n;
  return i < 0 ? i + n : i;
}

// Periodic wrap of a stencil index j = base - t of the per-site mesh kernels, whose base lies in
// [0, K + 1] and t in [0, p) with K >= 2 p: j is within [-K, 2K), so one conditional add or
// subtract suffices (no integer division); the final clamp keeps any input in bounds.
__device__ __forceinline__ int wrap_near(int j, int n) {
  j += j < 0 ? n : 0;
  j -= j >= n ? n : 0;
  return min(max(j, 0), n - 1);
}

// Row and column of stencil task t of a p x p tile: (t + 1/2) / p is never within 1 / (2p) of an
// integer, so the float product rounds to the exact quotient.
__device__ __forceinline__ int task_row(int t, float inv_p) { return (int)(((float)t + 0.5f) * inv_p); }

__device__ __forceinline__ void latch_error(int* status, int bit) { atomicOr(status, bit); }

// Programmatic dependent launch: kernels of the per-step chains are launched with the
// programmatic-serialization attribute (launch_pdl), so the next kernel's launch overlaps the
// previous one's exit; each such kernel first waits (griddepcontrol.wait) until its predecessor
// grid has completed and its memory is visible.  With the wait first, the order of memory effects
// is that of plain stream order.  No kernel triggers its dependents early: blocks of a successor
// resident while a long predecessor runs were measured to slow it.  Without a programmatic
// predecessor the wait returns at once.
__device__ __forceinline__ void pdl_enter() { asm volatile("griddepcontrol.wait;" ::: "memory"); }

template <typename... KArgs, typename... Args>
inline cudaError_t launch_pdl(void (*kernel)(KArgs...), dim3 grid, dim3 block, size_t smem, cudaStream_t st,
                              Args&&... args) {
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = grid;
  cfg.blockDim = block;
  cfg.dynamicSmemBytes = smem;
  cfg.stream = st;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  attr[0].val.programmaticStreamSerializationAllowed = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  return cudaLaunchKernelEx(&cfg, kernel, static_cast<KArgs>(args)...);
}

// Running sums in the working precision: float32 with a compensation term (TwoSum), float64 plain.
template <typename T> struct Acc;

template <> struct Acc<double> {
  double s = 0.0, c = 0.0;                     // c: an externally supplied correction (plain sums here)
  __device__ __forceinline__ void add(double x) { s += x; }
  __device__ __forceinline__ void warp_reduce() {
    s = warp_sum(s + c);
    c = 0.0;
  }
  __device__ __forceinline__ double value() const { return s + c; }
};

template <> struct Acc<float> {
  float s = 0.f, c = 0.f;
  __device__ __forceinline__ void add(float x) {
    const float t = s + x;
    const float bp = t - s;
    c += (s - (t - bp)) + (x - bp);
    s = t;
  }
  __device__ __forceinline__ void warp_reduce() {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      const float s2 = __shfl_xor_sync(0xffffffffu, s, o);
      const float c2 = __shfl_xor_sync(0xffffffffu, c, o);
      add(s2);
      c += c2;
    }
  }
  __device__ __forceinline__ double value() const { return (double)s + (double)c; }
};

template <typename T> __device__ __forceinline__ T warp_sum_t(T v) { return warp_sum(v); }

// block-wide sum of up to NV doubles held by lane 0 of every warp; thread 0 adds into dst[k].
template <int NV>
__device__ __forceinline__ void block_atomic_add(double (&v)[NV], double* const (&dst)[NV]) {
  __shared__ double red[NV][32];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, nw = blockDim.x >> 5;
  if (lane == 0)
    for (int k = 0; k < NV; ++k) red[k][warp] = v[k];
  __syncthreads();
  if (threadIdx.x == 0) {
    for (int k = 0; k < NV; ++k) {
      double s = 0;
      for (int w = 0; w < nw; ++w) s += red[k][w];
      if (dst[k] && s != 0.0) atomicAdd(dst[k], s);
    }
  }
}


// SPME mesh geometry shared by the mesh kernels.
struct SpmeGeom {
  int K[3];
  int P;
  double box[3];
  double kl[3];          // K_d / L_d
  long long Mr_s, Mc_s;
  int spl_off[3];        // axis offsets into the cell-origin tables
  int nc[3];             // real-space cell grid (flat cell index -> cell coordinates)
};

__device__ __forceinline__ int4 cell_coords(int flat, const SpmeGeom& sg) {
  return make_int4(flat / (sg.nc[2] * sg.nc[1]), (flat / sg.nc[2]) % sg.nc[1], flat % sg.nc[2], flat);
}

template <typename T>
__device__ __forceinline__ void site_weights(const typename Vec4<T>::type& p, const int4& cc, const SpmeGeom& sg,
                                             const int* __restrict__ splI, const T* __restrict__ splF, int lane,
                                             T (*w)[PMAX], T (*dw)[PMAX], int* i0) {
  if (lane < 3) {
    const T loc = lane == 0 ? p.x : (lane == 1 ? p.y : p.z);
    const int c = lane == 0 ? cc.x : (lane == 1 ? cc.y : cc.z);
    const int ti = sg.spl_off[lane] + c;
    const T u = splF[ti] + loc * (T)sg.kl[lane];
    const T fl = floor(u);
    T wl[PMAX], dl[PMAX];
    bspline<T>(u - fl, sg.P, wl, dl);
#pragma unroll
    for (int t = 0; t < PMAX; ++t) {
      w[lane][t] = wl[t];
      dw[lane][t] = dl[t];
    }
    i0[lane] = splI[ti] + (int)fl;
  }
  __syncwarp();
}

// B-spline weights of a batch of up to kSiteBatch electrolyte sites per warp: lane 3 s + d computes
// axis d of site s (s < nb), so one pass of the recursion serves nb sites instead of one (the
// stencil sweeps that follow use all 32 lanes per site).  Writes w / dw [s][d][t], the base mesh
// index b0 [s][d] and the charge q [s]; ends with __syncwarp.  Sites are taken in input order
// (l_tmp, l_cell), or with srt != nullptr in cell-sorted order (l_tmp then holds the sorted
// cell-local coordinates and srt the sorted -> input index map), which keeps neighbouring sites'
// stencils in the same cache lines.
constexpr int kSiteBatch = 10;
template <typename T>
__device__ __forceinline__ void batch_weights(int i0, int n, int nb, size_t kbase,
                                              const typename Vec4<T>::type* __restrict__ l_tmp,
                                              const int* __restrict__ l_cell, const SpmeGeom& sg,
                                              const int* __restrict__ splI, const T* __restrict__ splF, int lane,
                                              T (*w)[3][PMAX], T (*dw)[3][PMAX], int (*b0)[3], T* q,
                                              const int* __restrict__ srt = nullptr) {
  const int s = lane / 3, d = lane - 3 * s;
  if (s < nb && i0 + s < n) {
    const size_t k = kbase + i0 + s;
    const auto p = l_tmp[k];
    const int4 cc = cell_coords(l_cell[srt ? kbase + srt[k] : k], sg);
    const T loc = d == 0 ? p.x : (d == 1 ? p.y : p.z);
    const int c = d == 0 ? cc.x : (d == 1 ? cc.y : cc.z);
    const int ti = (d == 0 ? sg.spl_off[0] : (d == 1 ? sg.spl_off[1] : sg.spl_off[2])) + c;
    const T kl = (T)(d == 0 ? sg.kl[0] : (d == 1 ? sg.kl[1] : sg.kl[2]));
    const T u = splF[ti] + loc * kl;
    const T fl = floor(u);
    T wl[PMAX], dl[PMAX];
    bspline<T>(u - fl, sg.P, wl, dl);
#pragma unroll
    for (int t = 0; t < PMAX; ++t) {
      w[s][d][t] = wl[t];
      if (dw) dw[s][d][t] = dl[t];
    }
    b0[s][d] = splI[ti] + (int)fl;
    if (d == 0) q[s] = p.w;
  }
  __syncwarp();
}

// Electrolyte charges onto the mesh, in input order: k_bin's cell-local coordinates and cell index
// per site (no dependence on the sorted cell list, which is built concurrently on the side stream).

}  // namespace cpm

// Entry points implemented in cpm_step.cu, used by the build (Sv, checks).
namespace cpm {
// Blocks of the float64-heavy per-site kernels (S-apply finish, projections): 4 warps, so that a
// block's float64 reductions, on GB300's narrow float64 pipe, are spread over more SMs.
constexpr int FIN_THREADS = 128;
// q_raw = qpart + dpsi S v for one replica's rows, qpart cleared, with the projection sums
// (defined in cpm_step.cu; launched by the streaming and the packed S-apply).
__global__ void k_sapply_finish(int rows, double* __restrict__ qpart, const double* __restrict__ b,
                                const double* __restrict__ dpsi, const double* __restrict__ Sv,
                                const double* __restrict__ W, const double* __restrict__ c1,
                                double* __restrict__ qout, double* __restrict__ scal);
}  // namespace cpm
int cpm_internal_alloc_step_buffers(cpm_ctx* c);
int cpm_internal_static_scratch_setup();   // device address of cpm_step_charges_static's array
int cpm_internal_fft_setup(cpm_ctx* c);
int cpm_internal_convolve_own(cpm_ctx* c, int nrep, int energy_slot, cudaStream_t st);
cpm::SpmeGeom cpm_internal_spme_geom(const cpm_ctx* c);
int cpm_internal_brick_setup(cpm_ctx* c);
int cpm_internal_sym_setup(cpm_ctx* c);
bool cpm_internal_sym_fuse(const cpm_ctx* c);
int cpm_internal_sapply_sym(cpm_ctx* c, int blk, const float* xh, const float* xl, const double* b,
                            const double* dpsi, const double* Sv, const double* W, const double* c1, double* qout,
                            cudaStream_t st, bool fuse_sums);
int cpm_internal_spread_brick(cpm_ctx* c, int nrep, const void* l_loc, const float* qT, cudaStream_t st);
int cpm_internal_gather_f_brick(cpm_ctx* c, int nrep, const int* off, const void* l_loc, const double* dpsi,
                                double ff_over_lz, double slab_coef, double* F, cudaStream_t st);
