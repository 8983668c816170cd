// Per-step constant-potential electrostatics on the GPU (templated on the working precision T):
//
//   prepare   bin the electrolyte into the real-space cell grid (counting sort, cell-local coords)
//             k_bin, k_scan, k_scatter
//   charges   b = -(electrolyte potential at the electrode sites) (Eq. 3): real-space
//             Gaussian-point pairs (Eqs. 1-2 under the Ewald split, Sec. II.B; k_pair_cell,
//             k_pair_warp) + SPME (k_spread_*, FFT, k_influence, inverse FFT, k_gather_b),
//             then q = S (b + dpsi v) (k_sapply32 / 64 / stream / tc, cpm_sym.cu; the finite-field
//             v of Eq. 11, the doubled cell's of Eqs. 12-15) and the neutrality projection
//             (k_project, k_project_mirror; Eqs. 7-9 / 13-15)
//   forces    SPME of all charges + real-space pair forces (k_gather_f_*, k_pair_* with forces),
//             finite-field (Eqs. 10-11) / slab (Yeh-Berkowitz) terms, energies (k_energy_final:
//             Eq. 3 at the constrained optimum)
//
// Precision.  T = float is the mixed path.  GB300 issues float64 arithmetic at a small fraction of
// the float32 rate, so in the float kernels every per-lane sum is a compensated float32 sum
// (Knuth TwoSum), warp reductions combine (sum, error) pairs in float32, and float64 appears only
// in once-per-warp or once-per-site epilogues, in the input conversion and in the float64
// projection.  T = double is the plain float64 path: the same kernels with float64 throughout.
//
// Every launch goes to the caller's stream; nothing here allocates or synchronises the host.
#include "cpm_internal.cuh"

#include <algorithm>
#include <mutex>

namespace cpm {

constexpr unsigned FULL = 0xffffffffu;

struct CellGeom {
  int nc[3];
  int w[3];      // stencil widths 2 * sten + 1
  int sten[3];
  int nsten;
  int gz, ngz;   // pair kernels: z cells per block (a contiguous run of the sorted list), z groups
  double edge[3];
  double inv_edge[3];
  double box[3];
  double inv_box[3];
  double rc2;
  // float32 copies for the float32 pair kernels (no float64 conversion in the kernels: each costs
  // a float64-pipe instruction per warp on GB300)
  float alpha_f, rc2_f, edge_f[3];
};

// the field of the working precision: the float32 copy for float, the float64 value for double
template <typename T> __host__ __device__ __forceinline__ T prec_pick(double d, float f);
template <> __host__ __device__ __forceinline__ double prec_pick<double>(double d, float) { return d; }
template <> __host__ __device__ __forceinline__ float prec_pick<float>(double, float f) { return f; }



__device__ __forceinline__ double wrap_d(double x, double L, double invL) {
  double y = fma(-L, floor(x * invL), x);
  if (y >= L) y -= L;
  if (y < 0) y = 0;
  return y;
}

// ------------------------------------------------------------------------------------------
// prepare: counting sort of the electrolyte into cells
// ------------------------------------------------------------------------------------------
// Per site: wrap into the box, cell index, cell-local coordinates (float64 arithmetic, stored in
// the working precision) and the electrolyte dipole / charge-square sums.
template <typename T>
__global__ void __launch_bounds__(256) k_bin(const int* __restrict__ off, const double* __restrict__ xyzq, int cap,
                                             CellGeom g, double lz_phys, int* __restrict__ l_cell,
                                             int* __restrict__ l_count, typename Vec4<T>::type* __restrict__ l_tmp,
                                             int ncell, double* __restrict__ scal, int* __restrict__ status) {
  pdl_enter();
  using V4 = typename Vec4<T>::type;
  const int rep = blockIdx.y;
  const int o = off[rep];
  const int n_all = off[rep + 1] - o;
  const int n = min(n_all, cap);
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i == 0 && (n_all > cap || n_all < 0)) latch_error(status, DE_CAPACITY);
  double acc[2] = {0.0, 0.0};
  if (i < n) {
    const double4_32a s = reinterpret_cast<const double4_32a*>(xyzq)[o + i];
    double x = s.x, y = s.y, z = s.z, q = s.w;
    if (!(isfinite(x) && isfinite(y) && isfinite(z) && isfinite(q))) {
      latch_error(status, DE_NONFINITE);
      x = y = z = q = 0.0;
    } else if (!(z >= 0.0 && z < lz_phys)) {
      latch_error(status, DE_DOMAIN);
    }
    const double r[3] = {wrap_d(x, g.box[0], g.inv_box[0]), wrap_d(y, g.box[1], g.inv_box[1]),
                         wrap_d(z, g.box[2], g.inv_box[2])};
    int ci[3];
#pragma unroll
    for (int d = 0; d < 3; ++d) ci[d] = min(g.nc[d] - 1, max(0, (int)(r[d] * g.inv_edge[d])));
    const int flat = (ci[0] * g.nc[1] + ci[1]) * g.nc[2] + ci[2];
    l_cell[(size_t)rep * cap + i] = flat;
    atomicAdd(&l_count[(size_t)rep * ncell + flat], 1);
    V4 v;
    v.x = (T)fma(-(double)ci[0], g.edge[0], r[0]);
    v.y = (T)fma(-(double)ci[1], g.edge[1], r[1]);
    v.z = (T)fma(-(double)ci[2], g.edge[2], r[2]);
    v.w = (T)q;
    l_tmp[(size_t)rep * cap + i] = v;
    acc[0] = q * z;
    acc[1] = q * q;
  }
  acc[0] = warp_sum(acc[0]);
  acc[1] = warp_sum(acc[1]);
  double* const dst[2] = {scal + rep * NSCAL + S_QZ_ELYT, scal + rep * NSCAL + S_QQ_ELYT};
  block_atomic_add<2>(acc, dst);
}

// exclusive scan of the per-cell counts (one block per replica); counts become scatter cursors.
// Each warp owns a contiguous segment of 32 x SCAN_V cells per round: its lanes load the segment
// coalesced, all loads in flight at once, scan it 32 cells at a time with shuffles, then the warp
// totals are scanned across the block and added.
constexpr int SCAN_V = 16;
__global__ void __launch_bounds__(1024) k_scan(int* __restrict__ l_count, int* __restrict__ l_start, int ncell) {
  pdl_enter();
  const int rep = blockIdx.x;
  int* cnt = l_count + (size_t)rep * ncell;
  int* st = l_start + (size_t)rep * (ncell + 1);
  __shared__ int wtot[32];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nwarps = blockDim.x >> 5;
  int carry = 0;
  for (int base = 0; base < ncell; base += nwarps * 32 * SCAN_V) {
    const int seg = base + warp * 32 * SCAN_V;
    int c[SCAN_V];
#pragma unroll
    for (int j = 0; j < SCAN_V; ++j) {
      const int idx = seg + j * 32 + lane;
      c[j] = idx < ncell ? cnt[idx] : 0;
    }
    // c[j] becomes the exclusive prefix of element (j, lane) within the warp's segment
    int run = 0;
#pragma unroll
    for (int j = 0; j < SCAN_V; ++j) {
      int x = c[j];
#pragma unroll
      for (int o = 1; o < 32; o <<= 1) {
        const int u = __shfl_up_sync(FULL, x, o);
        if (lane >= o) x += u;
      }
      const int excl = run + x - c[j];
      run += __shfl_sync(FULL, x, 31);
      c[j] = excl;
    }
    if (lane == 0) wtot[warp] = run;
    __syncthreads();
    if (warp == 0) {
      int x = lane < nwarps ? wtot[lane] : 0;
      const int own = x;
#pragma unroll
      for (int o = 1; o < 32; o <<= 1) {
        const int u = __shfl_up_sync(FULL, x, o);
        if (lane >= o) x += u;
      }
      if (lane < nwarps) wtot[lane] = x - own;        // exclusive offset of each warp's segment
    }
    __syncthreads();
    const int off = carry + wtot[warp];
#pragma unroll
    for (int j = 0; j < SCAN_V; ++j) {
      const int idx = seg + j * 32 + lane;
      if (idx < ncell) {
        st[idx] = off + c[j];
        cnt[idx] = off + c[j];
      }
    }
    // the round's total: the last warp's offset plus its segment total
    const int last_off = wtot[nwarps - 1];
    __syncthreads();
    if (warp == nwarps - 1 && lane == 0) wtot[0] = last_off + run;
    __syncthreads();
    carry += wtot[0];
    __syncthreads();
  }
  if (threadIdx.x == 0) st[ncell] = carry;
}

template <typename T>
__global__ void __launch_bounds__(256) k_scatter(const int* __restrict__ off, int cap,
                                                 const int* __restrict__ l_cell,
                                                 const typename Vec4<T>::type* __restrict__ l_tmp,
                                                 int* __restrict__ cursor, int ncell, int* __restrict__ l_sorted,
                                                 typename Vec4<T>::type* __restrict__ l_loc) {
  pdl_enter();
  const int rep = blockIdx.y;
  const int n = min(off[rep + 1] - off[rep], cap);
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const size_t src = (size_t)rep * cap + i;
  const int flat = l_cell[src];
  const int pos = atomicAdd(&cursor[(size_t)rep * ncell + flat], 1);
  const size_t k = (size_t)rep * cap + pos;
  l_sorted[k] = i;
  l_loc[k] = l_tmp[src];
}

// Electrode charges in the working precision plus their float64 sums q z, q v, q^2, q_+.
template <typename T>
__global__ void __launch_bounds__(256) k_charge_prep(const double* __restrict__ q, int ne,
                                                     const double* __restrict__ ez, const double* __restrict__ ev,
                                                     const double* __restrict__ eplus, T* __restrict__ qT,
                                                     double* __restrict__ scal) {
  pdl_enter();
  const int rep = blockIdx.y;
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  double acc[4] = {0, 0, 0, 0};
  if (i < ne) {
    const double qi = q[(size_t)rep * ne + i];
    qT[(size_t)rep * ne + i] = (T)qi;
    acc[0] = qi * ez[i];
    acc[1] = qi * ev[i];
    acc[2] = qi * qi;
    acc[3] = qi * eplus[i];
  }
#pragma unroll
  for (int k = 0; k < 4; ++k) acc[k] = warp_sum(acc[k]);
  double* const dst[4] = {scal + rep * NSCAL + S_QZ_ELEC, scal + rep * NSCAL + S_QV_ELEC,
                          scal + rep * NSCAL + S_QQ_ELEC, scal + rep * NSCAL + S_QPLUS};
  block_atomic_add<4>(acc, dst);
}

// ------------------------------------------------------------------------------------------
// real-space pair sums: one block per target cell.  The block gathers the sources of every
// neighbour cell that can hold a point within r_c of the target cell into shared memory (image
// shift folded into the staged coordinates, charges attached), then each warp sweeps a share of
// the staged sources for one target.  Kernel per pair at distance r:
//   (erfc(alpha r) - erfc(beta r)) / r,  beta = 0 meaning a point source,
// and the force on the target  c_t c_s [kernel + 2/sqrt(pi)(alpha e^{-alpha^2 r^2} - beta e^{-beta^2 r^2})] d / r^2.
// ------------------------------------------------------------------------------------------
// Screened kernels of one pair at squared distance r2 (0 < r2 < rc^2): the potential factor
// pr = (erfc(alpha r) - erfc(beta r)) / r (beta = 0: point source, erfc(beta r) = 1 dropped) and the
// force factor fr = [pr + 2/sqrt(pi) (alpha e^{-alpha^2 r^2} - beta e^{-beta^2 r^2})] / r^2.
// float64: the library erfc and exp.  float32: erfc(x) = t P(t) e^{-x^2}, t = 1 / (1 + p x), P of
// degree 7 (Hastings' form, as in Abramowitz & Stegun 7.1.26, with coefficients fitted here to the
// relative error of erfc(x) e^{x^2} on 0 <= x <= 6.5 by erfc_fit.py: below 4e-8, under the float32
// rounding of the evaluation), so that one exponential serves both the potential and the force
// term and float32 pair sums carry no systematic approximation error.
template <typename T> struct PairMath;
template <> struct PairMath<double> {
  template <bool FORCE>
  __device__ __forceinline__ static void eval(double r2, double alpha, double beta, bool gauss, double& pr,
                                              double& fr) {
    const double r = sqrt(r2), ir = 1.0 / r;
    double num = erfc(alpha * r);
    double gxp = FORCE ? alpha * exp(-alpha * alpha * r2) : 0.0;
    if (gauss && beta * r < 6.5) {              // erfc(6.5) < 4e-20: below every float64 term
      num -= erfc(beta * r);
      if (FORCE) gxp -= beta * exp(-beta * beta * r2);
    }
    pr = num * ir;
    if (FORCE) fr = (pr + 1.1283791670955126 * gxp) * ir * ir;
  }
};
template <> struct PairMath<float> {
  __device__ __forceinline__ static float erfc_e(float x, float e) {     // e = exp(-x^2)
    const float t = __fdividef(1.0f, fmaf(0.42f, x, 1.0f));
    float poly = 7.600673979e-02f;
    poly = fmaf(poly, t, -3.450624826e-01f);
    poly = fmaf(poly, t, 4.849799364e-01f);
    poly = fmaf(poly, t, -1.730866602e-01f);
    poly = fmaf(poly, t, 2.924322982e-01f);
    poly = fmaf(poly, t, 1.871011462e-01f);
    poly = fmaf(poly, t, 2.408978217e-01f);
    poly = fmaf(poly, t, 2.367312164e-01f);
    return t * poly * e;
  }
  template <bool FORCE>
  __device__ __forceinline__ static void eval(float r2, float alpha, float beta, bool gauss, float& pr, float& fr) {
    const float ir = rsqrtf(r2), r = r2 * ir;
    const float ea = __expf(-alpha * alpha * r2);
    float num = erfc_e(alpha * r, ea);
    float gxp = alpha * ea;
    if (gauss && beta * r < 6.5f) {
      const float eb = __expf(-beta * beta * r2);
      num -= erfc_e(beta * r, eb);
      gxp -= beta * eb;
    }
    pr = num * ir;
    if (FORCE) fr = fmaf(1.1283791670955126f, gxp, pr) * ir * ir;
  }
};

struct PairSrc {
  const void* loc;          // cell-sorted cell-local coordinates (w = charge unless qT != nullptr)
  long long loc_stride;     // per-replica stride (0 = shared by all replicas)
  const int* start;         // [ncell + 1] cell starts
  long long start_stride;
  const int* sorted;        // sorted -> original index (electrode charge lookup)
  const void* qT;           // electrode charges [rep][q_stride] in the working precision, or nullptr
  int q_stride;
  double beta;              // second screening width: 0 = point source, else Gaussian kernel
  int slot;                 // energy slot receiving sum_t c_t phi_t, or -1
  float beta_f;             // float32 copy of beta (set by launch_pair)
};

struct CellPairTgt {
  const void* loc;          // cell-sorted cell-local coordinates (w = charge unless qT != nullptr)
  long long loc_stride;     // per replica (0: shared)
  const int* start;         // [ncell + 1] target cell starts
  long long start_stride;
  const int* sorted;        // sorted -> original index
  int n_fixed;              // per-replica stride of force (electrolyte: capacity) and phi_out (electrodes)
  const void* qT;           // electrode target charges [rep][n_fixed] in the working precision, or nullptr
  double* force;            // += KE c_t sum_s c_s g(r) d at [rep * n_fixed + original index][3], or nullptr
  double* phi_out;          // sum over set 0 of c_s kernel(r), [rep][n_fixed] original order, or nullptr
  double* field;            // FORCE: = KE sum_s c_s g(r) d over both sets, the force per unit target charge,
                            // at [rep * n_fixed + original index][3] (written, not added), or nullptr
  float* force_sorted;      // N3 kernels: forces added with float32 atomics at [rep * n_fixed + sorted index][3]
};

constexpr int PC_MAXT = 64;        // targets per pass of a block
constexpr int kPairSrcCap = 1024;  // sources staged per pass (dynamic shared memory)
constexpr int kPairSrcCapN3 = 1024; // the same for the third-law kernel
constexpr int PC_MAXSTEN = kMaxStencil;
constexpr int PC_THREADS = 256;
constexpr int PC_WARPS = PC_THREADS / 32;

// Lennard-Jones of an MD run, fused into the electrolyte-target force pass (LJ = true): the same
// staged sources and pair list within r_c serve both interactions.  Lorentz-Berthelot mixing,
// force-shifted at `cut` (<= r_c); electrolyte pairs count half their energy (seen from both ends).
struct PairLj {
  const int* type = nullptr;    // [offsets[n_rep]] per electrolyte site
  const int* off = nullptr;     // [n_rep + 1]
  int elec_type = -1;           // type of the electrode sources, -1: none
  double cut = 0.0;
  double sig_half[kLjMaxTypes] = {};
  double sqrt_eps[kLjMaxTypes] = {};
};

template <typename T> struct Vec2;
template <> struct Vec2<float> { using type = float2; };
template <> struct Vec2<double> { using type = double2; };

// N3 (electrolyte targets, float32, forces): Newton's third law for the point-point pairs of set 0,
// whose targets and sources are the same sites.  Set 0 is staged from the half stencil: the
// neighbour cells at a lexicographically positive offset (x, then y, then z) from the group's
// origin cell, which include the group's own cells; there a pair is taken once (source after
// target in the sorted order), so each unordered pair and each periodic image pair is evaluated
// once.  The source's
// reaction is added into a shared-memory accumulator of the staged source; after each batch the
// accumulators, and at the end the targets' own sums, are added with float32 atomics into
// t.force_sorted, indexed by sorted position (neighbouring sites, so the atomics of a block fall in
// few cache lines; float32 also keeps the conversions off GB300's narrow float64 pipe).  Set 1 (electrode sources) is as in the plain kernel.  The set-0 energy counts
// each pair twice, as the ordered sum of the plain kernel does.
template <typename T, bool FORCE, bool LJ = false, bool N3 = false>
__global__ void __launch_bounds__(PC_THREADS, N3 ? 4 : 0) k_pair_cell(const CellPairTgt t, const PairSrc s0, const PairSrc s1,
                                                          const CellGeom g, const double alpha_d, int src_cap,
                                                          double* __restrict__ scal, const PairLj lj) {
  pdl_enter();
  using V4 = typename Vec4<T>::type;
  using V2 = typename Vec2<T>::type;
  static_assert(!LJ || FORCE, "the Lennard-Jones pass computes forces");
  static_assert(!N3 || (FORCE && !LJ), "the third-law pass computes Coulomb forces");
  extern __shared__ __align__(32) unsigned char pc_dyn[];
  V4* src = reinterpret_cast<V4*>(pc_dyn);
  V2* src_lj = reinterpret_cast<V2*>(src + src_cap);          // LJ: (sigma / 2, sqrt eps) per staged source
  __shared__ V4 tpos[PC_MAXT];
  __shared__ V2 tlj[LJ ? PC_MAXT : 1];
  __shared__ T ilj[LJ ? 4 : 1][LJ ? PC_MAXT : 1];            // LJ force (3) and energy per item
  __shared__ T lpar[2][kLjMaxTypes];
  // per work item (target, part) of the current target batch, in the working precision:
  // compensated potential (sum, error) per source set, and the force sums
  __shared__ T ipot[2][PC_MAXT][2];
  __shared__ T ifrc[3][PC_MAXT];
  __shared__ int st_first[PC_MAXSTEN];
  __shared__ int st_pre[PC_MAXSTEN + 1];
  __shared__ T st_sh[3][PC_MAXSTEN];                // image / neighbour-cell shift of each stencil cell
  __shared__ int wq[PC_WARPS][128];             // per-warp ring of staged sources within r_c
  // per warp: the later part of a target whose first sweeps another warp owns (target or -1;
  // potential sum and error, force, Lennard-Jones force and energy)
  __shared__ int xs_tag[PC_WARPS];
  __shared__ T xs_v[PC_WARPS][9];
  // N3: reaction accumulator and sorted index of each staged source of set 0 (stored inverted for
  // sources outside the group's own cells: the ordering rule applies only inside them), and per
  // stencil cell whether it is one of the group's own cells
  __shared__ float n3_f[N3 ? 3 * kPairSrcCapN3 : 1];
  __shared__ int n3_gi[N3 ? kPairSrcCapN3 : 1];     // sorted index, bit-inverted (negative) outside the own cells
  __shared__ unsigned char n3_own[N3 ? PC_MAXSTEN : 1];

  const int rep = blockIdx.y;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  // this block's targets: the cells (cx, cy, cz .. cz + gzb - 1), contiguous in the sorted list;
  // coordinates are taken relative to the origin of cell (cx, cy, cz)
  const int czg = blockIdx.x % g.ngz, cy = (blockIdx.x / g.ngz) % g.nc[1], cx = blockIdx.x / (g.ngz * g.nc[1]);
  const int cz = czg * g.gz;
  const int gzb = min(g.gz, g.nc[2] - cz);
  const int cell = (cx * g.nc[1] + cy) * g.nc[2] + cz;
  const int* tst = t.start + rep * t.start_stride;
  const int t0 = tst[cell], t1 = tst[cell + gzb];
  if (t1 <= t0) return;                                    // whole block: empty cells
  if (tid < PC_WARPS) xs_tag[tid] = -1;                    // read only after the staging barriers
  const int wz = gzb + 2 * g.sten[2];                      // stencil extent in z for this group
  const int nsten = g.w[0] * g.w[1] * wz;
  const T alpha = prec_pick<T>(alpha_d, g.alpha_f);
  const T rc2 = prec_pick<T>(g.rc2, g.rc2_f);
  const T e0 = prec_pick<T>(g.edge[0], g.edge_f[0]), e1 = prec_pick<T>(g.edge[1], g.edge_f[1]),
          e2 = prec_pick<T>(g.edge[2], g.edge_f[2]);
  const V4* tl = (const V4*)t.loc + rep * t.loc_stride;
  const int* tso = t.sorted + rep * t.loc_stride;
  const T* tq = t.qT ? (const T*)t.qT + (size_t)rep * t.n_fixed : nullptr;
  const bool want_energy = s0.slot >= 0 || s1.slot >= 0;     // uniform over the block
  Acc<T> ea0, ea1;                  // sum_t c_t phi_t per source set, working precision, compensated
  const int lj_o = LJ ? lj.off[rep] : 0;
  const T ljc = (T)lj.cut, ljc2 = ljc * ljc, ljic = LJ ? T(1) / ljc : T(0);
  double elj = 0.0;                 // LJ energy of this block's targets
  if (LJ && tid == 0) {
#pragma unroll
    for (int k = 0; k < kLjMaxTypes; ++k) {
      lpar[0][k] = (T)lj.sig_half[k];
      lpar[1][k] = (T)lj.sqrt_eps[k];
    }
  }
  if (LJ) __syncthreads();

  for (int tb = t0; tb < t1; tb += PC_MAXT) {
    const int nt = min(PC_MAXT, t1 - tb);
    for (int k = tid; k < nt; k += PC_THREADS) {
      V4 p = tl[tb + k];
      if (tq) p.w = tq[tso[tb + k]];
      int j = 0;                                           // z cell of the target within the group
      while (j + 1 < gzb && tb + k >= tst[cell + j + 1]) ++j;
      p.z += (T)j * e2;
      tpos[k] = p;
      if (LJ) {
        const int ty = min(kLjMaxTypes - 1, max(0, lj.type[lj_o + tso[tb + k]]));
        V2 par;
        par.x = lpar[0][ty];
        par.y = lpar[1][ty];
        tlj[k] = par;
      }
    }
    for (int k = tid; k < nt; k += PC_THREADS) {
      ipot[0][k][0] = ipot[0][k][1] = ipot[1][k][0] = ipot[1][k][1] = T(0);
      ifrc[0][k] = ifrc[1][k] = ifrc[2][k] = T(0);
      if (LJ) ilj[0][k] = ilj[1][k] = ilj[2][k] = ilj[3][k] = T(0);
    }
    for (int set = 0; set < 2; ++set) {
      // fields of the selected source set, read into registers (no local copy of the parameters)
      const void* s_loc = set ? s1.loc : s0.loc;
      if (!s_loc) continue;
      const V4* sl = (const V4*)s_loc + rep * (set ? s1.loc_stride : s0.loc_stride);
      const int* sst = (set ? s1.start : s0.start) + rep * (set ? s1.start_stride : s0.start_stride);
      const void* s_q = set ? s1.qT : s0.qT;
      const T* sq = s_q ? (const T*)s_q + (size_t)rep * (set ? s1.q_stride : s0.q_stride) : nullptr;
      const int* s_sorted = set ? s1.sorted : s0.sorted;
      const int* s_sorted_r = s_sorted + rep * (set ? s1.loc_stride : s0.loc_stride);
      const T beta = set ? prec_pick<T>(s1.beta, s1.beta_f) : prec_pick<T>(s0.beta, s0.beta_f);
      const T ljw = set ? T(1) : T(0.5);      // electrolyte-electrolyte LJ pairs are seen from both ends
      const bool gauss = beta > T(0);
      // the potential sum of this set is wanted for an energy slot or (set 0) the potential output
      const bool need_pot = (set ? s1.slot : s0.slot) >= 0 || (set == 0 && t.phi_out != nullptr);
      __syncthreads();
      // ---- stencil cells whose box can hold a source within r_c of some point of this cell
      const float inv_w0 = 1.0f / (float)g.w[0], inv_w1 = 1.0f / (float)g.w[1];
      for (int si = tid; si < nsten; si += PC_THREADS) {
        // si = (dz' w1 + dy') w0 + dx' with small non-negative integers: the quotients by float
        // reciprocals are exact (si < 2^12)
        const int r1 = (int)(((float)si + 0.5f) * inv_w0);
        const int dx = si - r1 * g.w[0] - g.sten[0];
        const int r2 = (int)(((float)r1 + 0.5f) * inv_w1);
        const int dy = r1 - r2 * g.w[1] - g.sten[1];
        const int dz = r2 - g.sten[2];                      // -sten .. gzb - 1 + sten
        const int gapz = dz < 0 ? -dz - 1 : max(0, dz - gzb);
        const T gx = (T)max(0, abs(dx) - 1) * e0, gy = (T)max(0, abs(dy) - 1) * e1, gz = (T)gapz * e2;
        int c = 0, f = 0;
        // N3, set 0: the target cell and the neighbours at a lexicographically positive offset
        const bool half_ok = !N3 || set != 0 || dx > 0 || (dx == 0 && (dy > 0 || (dy == 0 && dz >= 0)));
        if (half_ok && gx * gx + gy * gy + gz * gz < rc2) {
          const int flat = (wrap_index(cx + dx, g.nc[0]) * g.nc[1] + wrap_index(cy + dy, g.nc[1])) * g.nc[2] +
                           wrap_index(cz + dz, g.nc[2]);
          f = sst[flat];
          c = sst[flat + 1] - f;
        }
        st_first[si] = f;
        st_pre[si + 1] = c;                 // counts, scanned below
        if (N3) n3_own[si] = (dx == 0 && dy == 0 && dz >= 0 && dz < gzb) ? 1 : 0;
        st_sh[0][si] = (T)dx * e0;
        st_sh[1][si] = (T)dy * e1;
        st_sh[2][si] = (T)dz * e2;
      }
      __syncthreads();
      // ---- inclusive scan of the counts (one warp, nsten <= PC_MAXSTEN)
      if (warp == 0) {
        int run = 0;
        for (int b = 0; b < nsten; b += 32) {
          const int k = b + lane;
          int v = k < nsten ? st_pre[k + 1] : 0;
#pragma unroll
          for (int o = 1; o < 32; o <<= 1) {
            const int u = __shfl_up_sync(FULL, v, o);
            if (lane >= o) v += u;
          }
          if (k < nsten) st_pre[k + 1] = run + v;
          run += __shfl_sync(FULL, v, 31);
        }
        if (lane == 0) st_pre[0] = 0;
      }
      __syncthreads();
      const int total = st_pre[nsten];
      const bool n3s = N3 && set == 0;
      for (int c0 = 0; c0 < total; c0 += src_cap) {
        const int ns = min(src_cap, total - c0);
        // ---- stage: k -> stencil entry by binary search over the prefix sums
        for (int k = tid; k < ns; k += PC_THREADS) {
          const int j = c0 + k;
          int lo = 0, hi = nsten;              // st_pre[lo] <= j < st_pre[hi]
          while (hi - lo > 1) {
            const int mid = (lo + hi) >> 1;
            if (st_pre[mid] <= j) lo = mid; else hi = mid;
          }
          const int gi = st_first[lo] + (j - st_pre[lo]);
          V4 p = sl[gi];
          p.x += st_sh[0][lo];
          p.y += st_sh[1][lo];
          p.z += st_sh[2][lo];
          if (sq) p.w = sq[s_sorted[gi]];
          src[k] = p;
          if (N3 && n3s) {
            n3_gi[k] = n3_own[lo] ? gi : ~gi;
            n3_f[3 * k + 0] = n3_f[3 * k + 1] = n3_f[3 * k + 2] = 0.f;
          }
          if (LJ) {
            const int ty = set ? lj.elec_type : min(kLjMaxTypes - 1, max(0, lj.type[lj_o + s_sorted_r[gi]]));
            V2 par;
            par.x = ty >= 0 ? lpar[0][ty] : T(0);
            par.y = ty >= 0 ? lpar[1][ty] : T(0);
            src_lj[k] = par;
          }
        }
        __syncthreads();
        // ---- compute: the work of the batch, nt targets x nch sweeps of 32 staged sources, is
        // split into equal contiguous ranges of (target, sweep) units, one per warp, so that every
        // warp reaches the barrier after the same work.  A warp takes the targets of its range in
        // turn; only its first target can start mid-way (the warp holding a target's first sweep
        // owns the target's slot, a later part goes to the warp's extra slot, added after the
        // barrier).  A cheap distance filter compacts the sources within r_c into a per-warp ring
        // (ballot + prefix), and the screened kernels run on 32 queued pairs at a time, so every
        // lane of the expensive part does useful work.  Per-lane running sums (compensated for the
        // potential) are reduced once per target and warp.
        int* ring = wq[warp];
        const int nch = (ns + 31) >> 5;
        const int units = nt * nch;
        const int u_end = ((warp + 1) * units) / PC_WARPS;
        for (int u = (warp * units) / PC_WARPS; u < u_end;) {
          const int ti = u / nch;
          const int kc0 = u - ti * nch, kc1 = min(nch, kc0 + (u_end - u));
          u += kc1 - kc0;
          const bool owner = kc0 == 0;
          const V4 tp = tpos[ti];
          Acc<T> pot;
          T fx = 0, fy = 0, fz = 0;
          T lx = 0, ly = 0, lz = 0, lu = 0;      // Lennard-Jones force and energy (LJ only)
          V2 tpar;
          if (LJ) tpar = tlj[ti];
          int head = 0, cnt = 0;                 // queued entries: ring[(head .. head + cnt) mod 128]
          auto consume = [&](int n) {
            if (lane < n) {
              const int idx = ring[(head + lane) & 127];
              const V4 sp = src[idx];
              const T dx = tp.x - sp.x, dy = tp.y - sp.y, dz = tp.z - sp.z;
              const T r2 = dx * dx + dy * dy + dz * dz;
              T pr, fr = T(0);
              PairMath<T>::template eval<FORCE>(r2, alpha, beta, gauss, pr, fr);
              if (need_pot) pot.add(sp.w * pr);
              if (FORCE) {
                fr *= sp.w;
                fx += fr * dx;
                fy += fr * dy;
                fz += fr * dz;
                if (N3 && n3s) {                 // the source's reaction, c_t c_s g(r) (-d)
                  const float rq = -(float)(tp.w * fr);
                  atomicAdd(&n3_f[3 * idx + 0], rq * (float)dx);
                  atomicAdd(&n3_f[3 * idx + 1], rq * (float)dy);
                  atomicAdd(&n3_f[3 * idx + 2], rq * (float)dz);
                }
              }
              if (LJ) {
                const V2 spar = src_lj[idx];
                const T eps = tpar.y * spar.y;
                if (r2 < ljc2 && eps > T(0)) {
                  const T sig = tpar.x + spar.x;
                  const T sg2 = sig * sig;
                  const T ir2 = T(1) / r2;
                  const T s2 = sg2 * ir2, s6 = s2 * s2 * s2;
                  const T c2 = sg2 * ljic * ljic, c6 = c2 * c2 * c2;
                  const T fc = T(24) * eps * (T(2) * c6 * c6 - c6) * ljic;   // force magnitude at the cutoff
                  const T r = sqrt(r2);
                  const T fl = T(24) * eps * ir2 * (T(2) * s6 * s6 - s6) - fc / r;
                  lx += fl * dx;
                  ly += fl * dy;
                  lz += fl * dz;
                  lu += ljw * (T(4) * eps * ((s6 * s6 - s6) - (c6 * c6 - c6)) + (r - ljc) * fc);
                }
              }
            }
            head = (head + n) & 127;
            cnt -= n;
            __syncwarp();
          };
          // two candidates per lane per step (64 staged sources), one ballot each: the ring's
          // bookkeeping is shared by both; at most 31 + 64 entries are queued before consuming
          const int kend = min(ns, kc1 * 32);
          const unsigned lt = (1u << lane) - 1u;
          // N3, set 0: in the group's own cells only sources after the target in the sorted order
          // (the group's cells are the half stencil's lowest cells of its own column)
          const int tgi = tb + ti;
          for (int kb = kc0 * 32; kb < kend; kb += 64) {
            const int k1 = kb + lane, k2 = kb + 32 + lane;
            bool h1 = false, h2 = false;
            if (k1 < kend) {
              const V4 sp = src[k1];
              const T dx = tp.x - sp.x, dy = tp.y - sp.y, dz = tp.z - sp.z;
              const T r2 = dx * dx + dy * dy + dz * dz;
              h1 = r2 < rc2 && r2 > T(0);
              if (N3 && n3s) {
                const int key = n3_gi[k1];
                h1 = h1 && (key < 0 || key > tgi);
              }
            }
            if (k2 < kend) {
              const V4 sp = src[k2];
              const T dx = tp.x - sp.x, dy = tp.y - sp.y, dz = tp.z - sp.z;
              const T r2 = dx * dx + dy * dy + dz * dz;
              h2 = r2 < rc2 && r2 > T(0);
              if (N3 && n3s) {
                const int key = n3_gi[k2];
                h2 = h2 && (key < 0 || key > tgi);
              }
            }
            const unsigned b1 = __ballot_sync(FULL, h1), b2 = __ballot_sync(FULL, h2);
            const int n1 = __popc(b1);
            if (h1) ring[(head + cnt + __popc(b1 & lt)) & 127] = k1;
            if (h2) ring[(head + cnt + n1 + __popc(b2 & lt)) & 127] = k2;
            cnt += n1 + __popc(b2);
            __syncwarp();
            if (cnt >= 32) consume(32);
            if (cnt >= 32) consume(32);
          }
          if (cnt > 0) consume(cnt);
          pot.warp_reduce();
          if (FORCE) {
            fx = warp_sum_t(fx);
            fy = warp_sum_t(fy);
            fz = warp_sum_t(fz);
          }
          if (LJ) {
            lx = warp_sum_t(lx);
            ly = warp_sum_t(ly);
            lz = warp_sum_t(lz);
            lu = warp_sum_t(lu);
          }
          if (lane == 0 && owner) {              // the target's slot belongs to its owner warp alone
            T* a = ipot[set][ti];
            const T t = a[0] + pot.s;
            const T bp = t - a[0];
            a[1] += ((a[0] - (t - bp)) + (pot.s - bp)) + pot.c;
            a[0] = t;
            if (FORCE) {
              ifrc[0][ti] += fx;
              ifrc[1][ti] += fy;
              ifrc[2][ti] += fz;
            }
            if (LJ) {
              ilj[0][ti] += lx;
              ilj[1][ti] += ly;
              ilj[2][ti] += lz;
              ilj[3][ti] += lu;
            }
          } else if (lane == 0) {                // a later part: the warp's extra slot
            xs_tag[warp] = ti;
            T* x = xs_v[warp];
            x[0] = pot.s;
            x[1] = pot.c;
            x[2] = fx;
            x[3] = fy;
            x[4] = fz;
            x[5] = lx;
            x[6] = ly;
            x[7] = lz;
            x[8] = lu;
          }
        }
        __syncthreads();
        // the warps' extra slots into the owners' slots (one thread: a target may have several)
        if (tid == 0) {
          for (int w = 0; w < PC_WARPS; ++w) {
            const int ti = xs_tag[w];
            if (ti < 0) continue;
            xs_tag[w] = -1;
            const T* x = xs_v[w];
            T* a = ipot[set][ti];
            const T t = a[0] + x[0];
            const T bp = t - a[0];
            a[1] += ((a[0] - (t - bp)) + (x[0] - bp)) + x[1];
            a[0] = t;
            ifrc[0][ti] += x[2];
            ifrc[1][ti] += x[3];
            ifrc[2][ti] += x[4];
            if (LJ) {
              ilj[0][ti] += x[5];
              ilj[1][ti] += x[6];
              ilj[2][ti] += x[7];
              ilj[3][ti] += x[8];
            }
          }
        }
        // N3: the staged sources' reactions of this batch (the same thread per staged slot as in
        // the staging loop, so the next batch's staging needs no extra barrier)
        if (N3 && n3s) {
          float* fs = t.force_sorted + 3 * (size_t)rep * t.n_fixed;
          const float ke = (float)KE;
          for (int k = tid; k < ns; k += PC_THREADS) {
            const float ax = n3_f[3 * k + 0], ay = n3_f[3 * k + 1], az = n3_f[3 * k + 2];
            if (ax != 0.f || ay != 0.f || az != 0.f) {
              const int v = n3_gi[k];
              float* o = fs + 3 * (size_t)(v >= 0 ? v : ~v);
              atomicAdd(o + 0, ke * ax);
              atomicAdd(o + 1, ke * ay);
              atomicAdd(o + 2, ke * az);
            }
          }
        }
      }
    }
    __syncthreads();
    // ---- outputs for this batch of targets (one thread per target): the parts are combined in
    // the working precision, then converted to float64 once
    for (int k = tid; k < nt; k += PC_THREADS) {
      const int orig = tso[tb + k];
      const double qt = (double)tpos[k].w;
      Acc<T> p0, p1;
      p0.s = ipot[0][k][0];
      p0.c = ipot[0][k][1];
      p1.s = ipot[1][k][0];
      p1.c = ipot[1][k][1];
      const T fx = FORCE ? ifrc[0][k] : T(0), fy = FORCE ? ifrc[1][k] : T(0), fz = FORCE ? ifrc[2][k] : T(0);
      if (t.phi_out) t.phi_out[(size_t)rep * t.n_fixed + orig] = p0.value();
      if (FORCE && t.field) {
        double* fo = t.field + 3 * ((size_t)rep * t.n_fixed + orig);
        fo[0] = KE * (double)fx;
        fo[1] = KE * (double)fy;
        fo[2] = KE * (double)fz;
      }
      if (want_energy) {
        const T ct = tpos[k].w;
        const T c0 = N3 ? T(2) * ct : ct;     // N3: set 0 saw each pair once; the slot wants both ends
        ea0.add(c0 * p0.s);
        ea0.c += c0 * p0.c;
        ea1.add(ct * p1.s);
        ea1.c += ct * p1.c;
      }
      if (N3) {                              // the target's own sums, beside the reactions it receives
        float* o = t.force_sorted + 3 * ((size_t)rep * t.n_fixed + tb + k);
        const float f = (float)KE * (float)tpos[k].w;
        atomicAdd(o + 0, f * (float)fx);
        atomicAdd(o + 1, f * (float)fy);
        atomicAdd(o + 2, f * (float)fz);
      }
      double ljf[3] = {0.0, 0.0, 0.0};
      if (LJ) {
        const T a0 = ilj[0][k], a1 = ilj[1][k], a2 = ilj[2][k], a3 = ilj[3][k];
        ljf[0] = (double)a0;
        ljf[1] = (double)a1;
        ljf[2] = (double)a2;
        elj += (double)a3;
      }
      if (FORCE && !N3 && t.force) {
        const size_t gi = (size_t)rep * t.n_fixed + orig;
        const double f = KE * qt;
        t.force[3 * gi + 0] += f * (double)fx + ljf[0];
        t.force[3 * gi + 1] += f * (double)fy + ljf[1];
        t.force[3 * gi + 2] += f * (double)fz + ljf[2];
      }
    }
    __syncthreads();
  }
  if (LJ) {
    __shared__ double ljred[PC_THREADS / 32];
    elj = warp_sum(elj);
    if (lane == 0) ljred[warp] = elj;
    __syncthreads();
    if (tid == 0) {
      double e = 0.0;
      for (int w = 0; w < PC_THREADS / 32; ++w) e += ljred[w];
      if (e != 0.0) atomicAdd(scal + rep * NSCAL + S_E_LJ, e);
    }
  }
  if (!want_energy) return;
  // block total in the working precision (compensated), one float64 atomic per slot
  __shared__ T ered[2][2][PC_THREADS / 32];
  ea0.warp_reduce();
  ea1.warp_reduce();
  if (lane == 0) {
    ered[0][0][warp] = ea0.s;
    ered[0][1][warp] = ea0.c;
    ered[1][0][warp] = ea1.s;
    ered[1][1][warp] = ea1.c;
  }
  __syncthreads();
  if (tid == 0) {
    Acc<T> a0, a1;
    for (int w = 0; w < PC_THREADS / 32; ++w) {
      a0.add(ered[0][0][w]);
      a0.c += ered[0][1][w];
      a1.add(ered[1][0][w]);
      a1.c += ered[1][1][w];
    }
    if (s0.slot >= 0) atomicAdd(scal + rep * NSCAL + s0.slot, a0.value());
    if (s1.slot >= 0) atomicAdd(scal + rep * NSCAL + s1.slot, a1.value());
  }
}

// Electrode-electrode real-space forces of the frozen electrode from the precomputed list
// (cpm_build: ee_ptr / ee_g): F_i += KE q_i sum_j q_j G_ij (mulq), or the field E_i += KE sum_j q_j G_ij
// when the force is formed later as q_i times the total field.  One warp per target row (grid-stride),
// grid.y = replica; each lane sums its share of the row in float32 (a few tens of terms), the
// lanes are combined in float64.  The list is streamed once per replica-step (16 bytes per pair);
// the charges are gathered through the caches.
__global__ void __launch_bounds__(256) k_ee_forces(const int* __restrict__ ptr, const float4* __restrict__ g, int ne,
                                                   const float* __restrict__ qT, double* __restrict__ f, int grp,
                                                   int mulq) {
  pdl_enter();
  const int rep = blockIdx.y;
  const int lane = threadIdx.x & 31;
  const float* q = qT + (size_t)rep * ne;
  const int nwarp = gridDim.x * (blockDim.x >> 5);
  const int warp = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
  // a warp takes grp (1..32) consecutive rows at a time; after each row's float32 reduction lane r
  // keeps row r's sums, and the float64 epilogue (a few instructions, costly on GB300's narrow
  // float64 pipe) then runs once per group, one lane per row
  for (int i0 = warp * grp; i0 < ne; i0 += nwarp * grp) {
    float mx = 0.f, my = 0.f, mz = 0.f;              // lane r: row i0 + r
    const int nrow = min(grp, ne - i0);
    for (int r = 0; r < nrow; ++r) {
      const int a = ptr[i0 + r], e = ptr[i0 + r + 1];
      Acc<float> sx, sy, sz;
      // four entries per lane per round: the list loads, then the charge gathers, all issued
      // before any is used
      for (int k0 = a + lane; k0 < e; k0 += 128) {
        float4 v[4];
#pragma unroll
        for (int u = 0; u < 4; ++u) {
          const int k = k0 + 32 * u;
          v[u] = k < e ? __ldcs(g + k) : make_float4(0.f, 0.f, 0.f, __int_as_float(0));
        }
        float qj[4];
#pragma unroll
        for (int u = 0; u < 4; ++u) qj[u] = __ldg(q + __float_as_int(v[u].w));
#pragma unroll
        for (int u = 0; u < 4; ++u) {
          sx.add(qj[u] * v[u].x);
          sy.add(qj[u] * v[u].y);
          sz.add(qj[u] * v[u].z);
        }
      }
      sx.warp_reduce();
      sy.warp_reduce();
      sz.warp_reduce();
      if (lane == r) {
        mx = sx.s + sx.c;
        my = sy.s + sy.c;
        mz = sz.s + sz.c;
      }
    }
    if (lane < nrow) {
      const int i = i0 + lane;
      const double c = mulq ? KE * (double)q[i] : KE;
      double* fi = f + 3 * ((size_t)rep * ne + i);
      fi[0] += c * (double)mx;
      fi[1] += c * (double)my;
      fi[2] += c * (double)mz;
    }
  }
}

// The same forces from the compressed list (lattice electrode): entry = j | t << 16, t indexing the
// table of distinct G vectors (cpm_build: ee_idx / ee_tab, the last entry zero), staged in shared
// memory; rows padded to a multiple of four entries, read as 16-byte chunks, four chunks in flight
// per lane.  LPR lanes share a row, 32 / LPR rows per pass of a warp; each lane sums the four
// products of a chunk in float32 and adds the chunks with compensation.  The list is streamed once
// per replica-step (4 bytes per pair); the charges are gathered through the caches.
template <int LPR>
__global__ void __launch_bounds__(256) k_ee_forces_tab(const int* __restrict__ ptr, const uint4* __restrict__ ent,
                                                       const float4* __restrict__ tab, int ntab, int ne,
                                                       const float* __restrict__ qT, double* __restrict__ f, int grp,
                                                       int mulq) {
  extern __shared__ float4 ee_sh[];
  constexpr int RPP = 32 / LPR;                        // rows per pass of a warp
  for (int k = threadIdx.x; k < ntab; k += blockDim.x) ee_sh[k] = tab[k];   // built once, not by the step
  pdl_enter();
  __syncthreads();
  const int rep = blockIdx.y;
  const int lane = threadIdx.x & 31, seg = lane / LPR, li = lane % LPR;
  const unsigned pz = (unsigned)(ntab - 1) << 16;     // j = 0 with the zero table entry
  const uint4 pad = make_uint4(pz, pz, pz, pz);
  const float* q = qT + (size_t)rep * ne;
  const int nwarp = gridDim.x * (blockDim.x >> 5);
  const int warp = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
  for (int i0 = warp * grp; i0 < ne; i0 += nwarp * grp) {
    const int nrow = min(grp, ne - i0);
    float mx = 0.f, my = 0.f, mz = 0.f;                // lane r: row i0 + r
    for (int r0 = 0; r0 < nrow; r0 += RPP) {
      const int r = r0 + seg;
      int a = 0, e = 0;                                // the row's 16-byte chunks
      if (r < nrow) {
        a = ptr[i0 + r] >> 2;
        e = ptr[i0 + r + 1] >> 2;
      }
      Acc<float> sx, sy, sz;
      for (int c0 = a + li; c0 < e; c0 += 4 * LPR) {
        uint4 v[4];
#pragma unroll
        for (int u = 0; u < 4; ++u) {
          const int c = c0 + u * LPR;
          v[u] = c < e ? __ldcs(ent + c) : pad;
        }
        float qj[16];
#pragma unroll
        for (int u = 0; u < 4; ++u) {
          qj[4 * u + 0] = __ldg(q + (v[u].x & 0xffffu));
          qj[4 * u + 1] = __ldg(q + (v[u].y & 0xffffu));
          qj[4 * u + 2] = __ldg(q + (v[u].z & 0xffffu));
          qj[4 * u + 3] = __ldg(q + (v[u].w & 0xffffu));
        }
#pragma unroll
        for (int u = 0; u < 4; ++u) {
          const unsigned w[4] = {v[u].x, v[u].y, v[u].z, v[u].w};
          float px = 0.f, py = 0.f, pz4 = 0.f;
#pragma unroll
          for (int h = 0; h < 4; ++h) {
            const float4 gv = ee_sh[w[h] >> 16];
            px = fmaf(qj[4 * u + h], gv.x, px);
            py = fmaf(qj[4 * u + h], gv.y, py);
            pz4 = fmaf(qj[4 * u + h], gv.z, pz4);
          }
          sx.add(px);
          sy.add(py);
          sz.add(pz4);
        }
      }
      // compensated sum over the row's LPR lanes (every lane of the segment ends with it)
#pragma unroll
      for (int o = LPR / 2; o > 0; o >>= 1) {
        const float x1 = __shfl_xor_sync(FULL, sx.s, o), x2 = __shfl_xor_sync(FULL, sx.c, o);
        const float y1 = __shfl_xor_sync(FULL, sy.s, o), y2 = __shfl_xor_sync(FULL, sy.c, o);
        const float z1 = __shfl_xor_sync(FULL, sz.s, o), z2 = __shfl_xor_sync(FULL, sz.c, o);
        sx.add(x1);
        sx.c += x2;
        sy.add(y1);
        sy.c += y2;
        sz.add(z1);
        sz.c += z2;
      }
      // segment g's row goes to lane r0 + g
#pragma unroll
      for (int g = 0; g < RPP; ++g) {
        const float vx = __shfl_sync(FULL, sx.s + sx.c, g * LPR);
        const float vy = __shfl_sync(FULL, sy.s + sy.c, g * LPR);
        const float vz = __shfl_sync(FULL, sz.s + sz.c, g * LPR);
        if (lane == r0 + g) {
          mx = vx;
          my = vy;
          mz = vz;
        }
      }
    }
    if (lane < nrow) {                                 // float64 epilogue once per group of rows
      const int i = i0 + lane;
      const double c = mulq ? KE * (double)q[i] : KE;
      double* fi = f + 3 * ((size_t)rep * ne + i);
      fi[0] += c * (double)mx;
      fi[1] += c * (double)my;
      fi[2] += c * (double)mz;
    }
  }
}

// Warp-per-target variant of the real-space pair kernels (same inputs and outputs as k_pair_cell).
// A warp takes one target at a time (grid-stride over the cell-sorted targets): it lists the
// stencil cells whose box lies within r_c of the target point itself (tighter than the cell-to-cell
// test of k_pair_cell), scans their source counts, then sweeps the candidates 32 at a time straight
// from global memory (L1 / L2: neighbouring warps read the same cells), compacting those within r_c
// into a per-warp ring for the screened kernels.  No block-wide staging, no block barriers until
// the final energy reduction.
constexpr int PW_THREADS = 256;
constexpr int PW_WARPS = PW_THREADS / 32;

// per-warp shared memory: stencil prefix [ns + 1], first source [ns], packed offsets [ns], ring
template <typename T>
__host__ __device__ constexpr size_t pw_warp_bytes(int ns) {
  // multiple of 32 bytes, so that every warp's ring of (32-byte float64) positions stays aligned
  return ((sizeof(int) * (3 * (size_t)ns + 1) + 64 * (sizeof(typename Vec4<T>::type) +
                                                      sizeof(typename Vec2<T>::type))) + 31) & ~(size_t)31;
}

template <typename T, bool FORCE, bool LJ = false>
__global__ void __launch_bounds__(PW_THREADS) k_pair_warp(const CellPairTgt t, const PairSrc s0, const PairSrc s1,
                                                          const CellGeom g, const double alpha_d, double* __restrict__ scal,
                                                          const PairLj lj) {
  pdl_enter();
  using V4 = typename Vec4<T>::type;
  using V2 = typename Vec2<T>::type;
  static_assert(!LJ || FORCE, "the Lennard-Jones pass computes forces");
  extern __shared__ __align__(32) unsigned char pw_dyn[];
  __shared__ T lpar[2][kLjMaxTypes];
  __shared__ double ered[3][PW_WARPS];
  const int rep = blockIdx.y;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int ns = g.nsten;
  unsigned char* wbase = pw_dyn + (size_t)warp * pw_warp_bytes<T>(ns);
  V4* rsrc = reinterpret_cast<V4*>(wbase);                              // ring: source positions
  V2* rlj = reinterpret_cast<V2*>(rsrc + 64);                           // ring: LJ parameters
  int* wpre = reinterpret_cast<int*>(rlj + 64);                         // [ns + 1]
  int* wfirst = wpre + ns + 1;                                          // [ns]
  int* wdoff = wfirst + ns;                                             // [ns] packed (dx, dy, dz)
  if (LJ && tid == 0) {
#pragma unroll
    for (int k = 0; k < kLjMaxTypes; ++k) {
      lpar[0][k] = (T)lj.sig_half[k];
      lpar[1][k] = (T)lj.sqrt_eps[k];
    }
  }
  __syncthreads();
  const int ncell = g.nc[0] * g.nc[1] * g.nc[2];
  const int* tst = t.start + rep * t.start_stride;
  const int n_t = tst[ncell];
  const V4* tl = (const V4*)t.loc + rep * t.loc_stride;
  const int* tso = t.sorted + rep * t.loc_stride;
  const T* tq = t.qT ? (const T*)t.qT + (size_t)rep * t.n_fixed : nullptr;
  const bool want_energy = s0.slot >= 0 || s1.slot >= 0;
  const T alpha = prec_pick<T>(alpha_d, g.alpha_f);
  const T rc2 = prec_pick<T>(g.rc2, g.rc2_f);
  const T e0 = prec_pick<T>(g.edge[0], g.edge_f[0]), e1 = prec_pick<T>(g.edge[1], g.edge_f[1]),
          e2 = prec_pick<T>(g.edge[2], g.edge_f[2]);
  const int lj_o = LJ ? lj.off[rep] : 0;
  const T ljc = (T)lj.cut, ljc2 = ljc * ljc, ljic = LJ ? T(1) / ljc : T(0);
  Acc<T> ea0, ea1;                                                      // lane 0 of each warp
  double elj = 0.0;
  for (int k = blockIdx.x * PW_WARPS + warp; k < n_t; k += gridDim.x * PW_WARPS) {
    // the target's cell: the last c with tst[c] <= k
    int lo = 0, hi = ncell;
    while (hi - lo > 1) {
      const int mid = (lo + hi) >> 1;
      if (tst[mid] <= k) lo = mid; else hi = mid;
    }
    const int cell = lo;
    const int cz = cell % g.nc[2], cy = (cell / g.nc[2]) % g.nc[1], cx = cell / (g.nc[2] * g.nc[1]);
    V4 tp = tl[k];
    const int orig = tso[k];
    if (tq) tp.w = tq[orig];
    V2 tpar;
    if (LJ) {
      const int ty = min(kLjMaxTypes - 1, max(0, lj.type[lj_o + orig]));
      tpar.x = lpar[0][ty];
      tpar.y = lpar[1][ty];
    }
    Acc<T> pot[2];
    T fx = 0, fy = 0, fz = 0;
    T lx = 0, ly = 0, lz = 0, lu = 0;
    for (int set = 0; set < 2; ++set) {
      const void* s_loc = set ? s1.loc : s0.loc;
      if (!s_loc) continue;
      const long long s_ls = set ? s1.loc_stride : s0.loc_stride;
      const V4* sl = (const V4*)s_loc + rep * s_ls;
      const int* sst = (set ? s1.start : s0.start) + rep * (set ? s1.start_stride : s0.start_stride);
      const void* s_q = set ? s1.qT : s0.qT;
      const T* sq = s_q ? (const T*)s_q + (size_t)rep * (set ? s1.q_stride : s0.q_stride) : nullptr;
      const int* s_sorted = set ? s1.sorted : s0.sorted;
      const int* s_sorted_r = s_sorted + rep * s_ls;
      const T beta = set ? prec_pick<T>(s1.beta, s1.beta_f) : prec_pick<T>(s0.beta, s0.beta_f);
      const bool gauss = beta > T(0);
      const T ljw = set ? T(1) : T(0.5);
      // ---- stencil cells within r_c of the target point, and their source counts
      int run = 0;
      for (int b = 0; b < ns; b += 32) {
        const int si = b + lane;
        int cnt = 0, f = 0, pack = 0;
        if (si < ns) {
          const int dx = si % g.w[0] - g.sten[0];
          const int r1 = si / g.w[0];
          const int dy = r1 % g.w[1] - g.sten[1];
          const int dz = r1 / g.w[1] - g.sten[2];
          const T bx = (T)dx * e0, by = (T)dy * e1, bz = (T)dz * e2;
          const T qx = fmax(T(0), fmax(bx - tp.x, tp.x - (bx + e0)));
          const T qy = fmax(T(0), fmax(by - tp.y, tp.y - (by + e1)));
          const T qz = fmax(T(0), fmax(bz - tp.z, tp.z - (bz + e2)));
          if (qx * qx + qy * qy + qz * qz < rc2) {
            const int flat = (wrap_index(cx + dx, g.nc[0]) * g.nc[1] + wrap_index(cy + dy, g.nc[1])) * g.nc[2] +
                             wrap_index(cz + dz, g.nc[2]);
            f = sst[flat];
            cnt = sst[flat + 1] - f;
          }
          pack = ((dx + 128) << 16) | ((dy + 128) << 8) | (dz + 128);
        }
        int v = cnt;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
          const int u = __shfl_up_sync(FULL, v, o);
          if (lane >= o) v += u;
        }
        if (si < ns) {
          wpre[si + 1] = run + v;
          wfirst[si] = f;
          wdoff[si] = pack;
        }
        run += __shfl_sync(FULL, v, 31);
      }
      if (lane == 0) wpre[0] = 0;
      __syncwarp();
      const int total = run;
      // ---- candidates 32 at a time; those within r_c go to the ring
      int head = 0, cnt = 0;
      auto consume = [&](int n) {
        if (lane < n) {
          const int slot = (head + lane) & 63;
          const V4 sp = rsrc[slot];
          const T dx = tp.x - sp.x, dy = tp.y - sp.y, dz = tp.z - sp.z;
          const T r2 = dx * dx + dy * dy + dz * dz;
          T pr, fr = T(0);
          PairMath<T>::template eval<FORCE>(r2, alpha, beta, gauss, pr, fr);
          pot[set].add(sp.w * pr);
          if (FORCE) {
            fr *= sp.w;
            fx += fr * dx;
            fy += fr * dy;
            fz += fr * dz;
          }
          if (LJ) {
            const V2 spar = rlj[slot];
            const T eps = tpar.y * spar.y;
            if (r2 < ljc2 && eps > T(0)) {
              const T sig = tpar.x + spar.x;
              const T sg2 = sig * sig;
              const T ir2 = T(1) / r2;
              const T s2 = sg2 * ir2, s6 = s2 * s2 * s2;
              const T c2 = sg2 * ljic * ljic, c6 = c2 * c2 * c2;
              const T fc = T(24) * eps * (T(2) * c6 * c6 - c6) * ljic;
              const T r = sqrt(r2);
              const T fl = T(24) * eps * ir2 * (T(2) * s6 * s6 - s6) - fc / r;
              lx += fl * dx;
              ly += fl * dy;
              lz += fl * dz;
              lu += ljw * (T(4) * eps * ((s6 * s6 - s6) - (c6 * c6 - c6)) + (r - ljc) * fc);
            }
          }
        }
        head = (head + n) & 63;
        cnt -= n;
        __syncwarp();
      };
      for (int jb = 0; jb < total; jb += 32) {
        const int j = jb + lane;
        bool hit = false;
        V4 p;
        V2 par;
        if (j < total) {
          int a = 0, bnd = ns;                                          // wpre[a] <= j < wpre[bnd]
          while (bnd - a > 1) {
            const int mid = (a + bnd) >> 1;
            if (wpre[mid] <= j) a = mid; else bnd = mid;
          }
          const int gi = wfirst[a] + (j - wpre[a]);
          const int pk = wdoff[a];
          p = sl[gi];
          p.x += (T)(((pk >> 16) & 255) - 128) * e0;
          p.y += (T)(((pk >> 8) & 255) - 128) * e1;
          p.z += (T)((pk & 255) - 128) * e2;
          const T dx = tp.x - p.x, dy = tp.y - p.y, dz = tp.z - p.z;
          const T r2 = dx * dx + dy * dy + dz * dz;
          hit = r2 < rc2 && r2 > T(0);
          if (hit && sq) p.w = sq[s_sorted[gi]];
          if (LJ && hit) {
            const int ty = set ? lj.elec_type : min(kLjMaxTypes - 1, max(0, lj.type[lj_o + s_sorted_r[gi]]));
            par.x = ty >= 0 ? lpar[0][ty] : T(0);
            par.y = ty >= 0 ? lpar[1][ty] : T(0);
          }
        }
        const unsigned bal = __ballot_sync(FULL, hit);
        if (hit) {
          const int slot = (head + cnt + __popc(bal & ((1u << lane) - 1u))) & 63;
          rsrc[slot] = p;
          if (LJ) rlj[slot] = par;
        }
        cnt += __popc(bal);
        __syncwarp();
        if (cnt >= 32) consume(32);
      }
      if (cnt > 0) consume(cnt);
      __syncwarp();
    }
    // ---- this target's outputs
    pot[0].warp_reduce();
    pot[1].warp_reduce();
    if (FORCE) {
      fx = warp_sum_t(fx);
      fy = warp_sum_t(fy);
      fz = warp_sum_t(fz);
    }
    if (LJ) {
      lx = warp_sum_t(lx);
      ly = warp_sum_t(ly);
      lz = warp_sum_t(lz);
      lu = warp_sum_t(lu);
    }
    if (lane == 0) {
      if (t.phi_out) t.phi_out[(size_t)rep * t.n_fixed + orig] = pot[0].value();
      if (FORCE && t.field) {
        double* fo = t.field + 3 * ((size_t)rep * t.n_fixed + orig);
        fo[0] = KE * (double)fx;
        fo[1] = KE * (double)fy;
        fo[2] = KE * (double)fz;
      }
      if (want_energy) {
        const T ct = tp.w;
        ea0.add(ct * pot[0].s);
        ea0.c += ct * pot[0].c;
        ea1.add(ct * pot[1].s);
        ea1.c += ct * pot[1].c;
      }
      if (LJ) elj += (double)lu;
      if (FORCE && t.force) {
        const size_t gi = (size_t)rep * t.n_fixed + orig;
        const double f = KE * (double)tp.w;
        t.force[3 * gi + 0] += f * (double)fx + (LJ ? (double)lx : 0.0);
        t.force[3 * gi + 1] += f * (double)fy + (LJ ? (double)ly : 0.0);
        t.force[3 * gi + 2] += f * (double)fz + (LJ ? (double)lz : 0.0);
      }
    }
    __syncwarp();
  }
  // ---- block totals: one float64 atomic per energy slot per block
  if (!want_energy && !LJ) return;
  if (lane == 0) {
    ered[0][warp] = ea0.value();
    ered[1][warp] = ea1.value();
    ered[2][warp] = elj;
  }
  __syncthreads();
  if (tid == 0) {
    double a0 = 0.0, a1 = 0.0, a2 = 0.0;
    for (int w = 0; w < PW_WARPS; ++w) {
      a0 += ered[0][w];
      a1 += ered[1][w];
      a2 += ered[2][w];
    }
    if (s0.slot >= 0 && a0 != 0.0) atomicAdd(scal + rep * NSCAL + s0.slot, a0);
    if (s1.slot >= 0 && a1 != 0.0) atomicAdd(scal + rep * NSCAL + s1.slot, a1);
    if (LJ && a2 != 0.0) atomicAdd(scal + rep * NSCAL + S_E_LJ, a2);
  }
}

// ------------------------------------------------------------------------------------------
// SPME: charge assignment, influence function, interpolation (cardinal B-splines of order P)
// ------------------------------------------------------------------------------------------
// B-spline weights of one cell-sorted electrolyte site into per-warp shared memory (lanes 0-2
// handle axes x, y, z).  Its mesh coordinate u = (cell origin) + (local offset) K/L uses the
// per-cell integer / fraction tables, so only the small local part is formed in precision T.
template <typename T>
__device__ __forceinline__ void spread_elyt_sites(int bx, int nbx, int nb, const int* __restrict__ off, int cap,
                                                  const SpmeGeom sg,
                                                  const typename Vec4<T>::type* __restrict__ l_tmp,
                                                  const int* __restrict__ l_cell, const int* __restrict__ splI,
                                                  const T* __restrict__ splF, T* __restrict__ mesh,
                                                  const int* __restrict__ srt = nullptr) {
  __shared__ T sw[8][kSiteBatch][3][PMAX];
  __shared__ int si0[8][kSiteBatch][3];
  __shared__ T sq[8][kSiteBatch];
  const int rep = blockIdx.y;
  const int n = min(off[rep + 1] - off[rep], cap);
  const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5;
  const int P = sg.P, K1 = sg.K[0], K2 = sg.K[1], K3 = sg.K[2];
  const float inv_p = 1.0f / (float)P;
  // the lane's (y, z) stencil tasks (lane and lane + 32), computed once: the int <-> float
  // conversions of the row index stay out of the per-site loops
  const int ty0 = task_row(lane, inv_p), tz0 = lane - ty0 * P;
  const int ty1 = task_row(lane + 32, inv_p), tz1 = lane + 32 - ty1 * P;
  T* m = mesh + (size_t)rep * sg.Mr_s;
  const int nw = (nbx * blockDim.x) >> 5;
  const int first = (bx * blockDim.x + threadIdx.x) >> 5;
  // warp-batches of nb consecutive sites: the weights of the batch in one pass, then each site's stencil
  for (int i0 = first * nb; i0 < n; i0 += nw * nb) {
    batch_weights<T>(i0, n, nb, (size_t)rep * cap, l_tmp, l_cell, sg, splI, splF, lane, sw[wib], nullptr, si0[wib],
                     sq[wib], srt);
    const int cnt = min(nb, n - i0);
    for (int si = 0; si < cnt; ++si) {
      const T qv = sq[wib][si];
      const int* b0 = si0[wib][si];
      for (int task = lane; task < P * P; task += 32) {
        const int ty = task < 32 ? ty0 : ty1, tz = task < 32 ? tz0 : tz1;
        const int gy = wrap_near(b0[1] - ty, K2), gz = wrap_near(b0[2] - tz, K3);
        const T wyz = qv * sw[wib][si][1][ty] * sw[wib][si][2][tz];
        for (int tx = 0; tx < P; ++tx) {
          const int gx = wrap_near(b0[0] - tx, K1);
          atomicAdd(&m[((size_t)gx * K2 + gy) * K3 + gz], sw[wib][si][0][tx] * wyz);
        }
      }
    }
    __syncwarp();
  }
}

// Electrode charges onto the mesh through the fixed stencils.
template <typename T>
__device__ __forceinline__ void spread_elec_sites(int bx, int nbx, const T* __restrict__ qT, int ne,
                                                  const int4* __restrict__ base, const T* __restrict__ th,
                                                  const SpmeGeom sg, T* __restrict__ mesh) {
  const int rep = blockIdx.y;
  const int lane = threadIdx.x & 31;
  const int P = sg.P, K1 = sg.K[0], K2 = sg.K[1], K3 = sg.K[2];
  const float inv_p = 1.0f / (float)P;
  // the lane's (y, z) stencil tasks (lane and lane + 32), computed once: the int <-> float
  // conversions of the row index stay out of the per-site loops
  const int ty0 = task_row(lane, inv_p), tz0 = lane - ty0 * P;
  const int ty1 = task_row(lane + 32, inv_p), tz1 = lane + 32 - ty1 * P;
  T* m = mesh + (size_t)rep * sg.Mr_s;
  const T* qr = qT + (size_t)rep * ne;
  for (int i = (bx * blockDim.x + threadIdx.x) >> 5; i < ne; i += (nbx * blockDim.x) >> 5) {
    const T qi = qr[i];
    const int4 b = base[i];
    const T* w = th + (size_t)i * 3 * PMAX;
    for (int task = lane; task < P * P; task += 32) {
      const int ty = task < 32 ? ty0 : ty1, tz = task < 32 ? tz0 : tz1;
      const int gy = wrap_near(b.y - ty, K2), gz = wrap_near(b.z - tz, K3);
      const T wyz = qi * w[PMAX + ty] * w[2 * PMAX + tz];
      for (int tx = 0; tx < P; ++tx) {
        const int gx = wrap_near(b.x - tx, K1);
        atomicAdd(&m[((size_t)gx * K2 + gy) * K3 + gz], w[tx] * wyz);
      }
    }
  }
}

// rho^(m) *= G(m) on the half spectrum; optionally E_recip += 1/2 sum_m G |rho^(m)|^2 (full spectrum).
// Electrolyte charges onto the mesh (warp per site, input order), electrode charges through their
// fixed stencils, and both in one launch (blocks [0, nb_elyt) take the electrolyte).
template <typename T>
__global__ void __launch_bounds__(256) k_spread_elyt(int nb, const int* __restrict__ off, int cap, SpmeGeom sg,
                                                     const typename Vec4<T>::type* __restrict__ l_tmp,
                                                     const int* __restrict__ l_cell, const int* __restrict__ splI,
                                                     const T* __restrict__ splF, T* __restrict__ mesh) {
  pdl_enter();
  spread_elyt_sites<T>(blockIdx.x, gridDim.x, nb, off, cap, sg, l_tmp, l_cell, splI, splF, mesh);
}

template <typename T>
__global__ void __launch_bounds__(256) k_spread_elec(const T* __restrict__ qT, int ne, const int4* __restrict__ base,
                                                     const T* __restrict__ th, SpmeGeom sg, T* __restrict__ mesh) {
  spread_elec_sites<T>(blockIdx.x, gridDim.x, qT, ne, base, th, sg, mesh);
}

template <typename T>
__global__ void __launch_bounds__(256) k_spread_all(int nb_elyt, int nb, const int* __restrict__ off, int cap,
                                                    SpmeGeom sg,
                                                    const typename Vec4<T>::type* __restrict__ l_tmp,
                                                    const int* __restrict__ l_cell, const int* __restrict__ splI,
                                                    const T* __restrict__ splF, const T* __restrict__ qT, int ne,
                                                    const int4* __restrict__ base, const T* __restrict__ th,
                                                    T* __restrict__ mesh, const int* __restrict__ srt) {
  pdl_enter();
  if ((int)blockIdx.x < nb_elyt)
    spread_elyt_sites<T>(blockIdx.x, nb_elyt, nb, off, cap, sg, l_tmp, l_cell, splI, splF, mesh, srt);
  else
    spread_elec_sites<T>(blockIdx.x - nb_elyt, gridDim.x - nb_elyt, qT, ne, base, th, sg, mesh);
}

template <typename T, typename T2>
__global__ void __launch_bounds__(256) k_influence(T2* __restrict__ spec, const T* __restrict__ G, long long Mc,
                                                   long long Mc_s, int K3h, int K3, int energy_slot,
                                                   double* __restrict__ scal) {
  pdl_enter();
  const bool energy = energy_slot >= 0;
  const int rep = blockIdx.y;
  T2* c = spec + (size_t)rep * Mc_s;
  Acc<T> e;
  for (long long k = blockIdx.x * (long long)blockDim.x + threadIdx.x; k < Mc; k += (long long)gridDim.x * blockDim.x) {
    T2 v = c[k];
    const T g = G[k];
    if (energy) {
      const int n3 = (int)(k % K3h);
      const T wgt = (n3 == 0 || 2 * n3 == K3) ? T(0.5) : T(1);
      e.add(wgt * g * (v.x * v.x + v.y * v.y));
    }
    v.x *= g;
    v.y *= g;
    c[k] = v;
  }
  if (energy) {
    e.warp_reduce();
    double acc[1] = {e.value()};
    double* const dst[1] = {scal + rep * NSCAL + energy_slot};
    block_atomic_add<1>(acc, dst);
  }
}

// b_i = -(KE phi_real_i + phi_mesh_i) (- KE 4 pi / V z_i sum_j Q_j Z_j for the slab), one warp per site,
// written to b (row stride ldb); with b32 != nullptr also the float32 split b = hi + lo
// (hi = fl(b), lo = fl(b - hi)) for the mixed-precision S-apply, halves of length ldx.

template <typename T>
__global__ void __launch_bounds__(256) k_gather_b(const T* __restrict__ phi, int ne, const int4* __restrict__ base,
                                                  const T* __restrict__ th, SpmeGeom sg,
                                                  const double* __restrict__ phi_real, const double* __restrict__ ez,
                                                  double slab_coef, const double* __restrict__ scal,
                                                  double* __restrict__ b, float* __restrict__ b32, int ldx,
                                                  int ldb, int grp) {
  pdl_enter();
  const int rep = blockIdx.y;
  const int lane = threadIdx.x & 31;
  const int P = sg.P, K1 = sg.K[0], K2 = sg.K[1], K3 = sg.K[2];
  const float inv_p = 1.0f / (float)P;
  // the lane's (y, z) stencil tasks (lane and lane + 32), computed once: the int <-> float
  // conversions of the row index stay out of the per-site loops
  const int ty0 = task_row(lane, inv_p), tz0 = lane - ty0 * P;
  const int ty1 = task_row(lane + 32, inv_p), tz1 = lane + 32 - ty1 * P;
  const T* m = phi + (size_t)rep * sg.Mr_s;
  const int nwarp = (gridDim.x * blockDim.x) >> 5;
  // grp (1..32) consecutive sites per warp: each site's stencil over the lanes (compensated), lane s
  // keeping site s's sum; the float64 epilogue once per group, one lane per site
  for (int i0 = ((blockIdx.x * blockDim.x + threadIdx.x) >> 5) * grp; i0 < ne; i0 += nwarp * grp) {
    const int ns = min(grp, ne - i0);
    T ks = 0, kc = 0;
    for (int si = 0; si < ns; ++si) {
      const int i = i0 + si;
      const int4 bs = base[i];
      const T* w = th + (size_t)i * 3 * PMAX;
      Acc<T> acc;
      for (int task = lane; task < P * P; task += 32) {
        const int ty = task < 32 ? ty0 : ty1, tz = task < 32 ? tz0 : tz1;
        const int gy = wrap_near(bs.y - ty, K2), gz = wrap_near(bs.z - tz, K3);
        T ph[PMAX];
#pragma unroll
        for (int tx = 0; tx < PMAX; ++tx)
          ph[tx] = tx < P ? m[((size_t)wrap_near(bs.x - tx, K1) * K2 + gy) * K3 + gz] : T(0);
        T sx = 0;
#pragma unroll
        for (int tx = 0; tx < PMAX; ++tx)
          if (tx < P) sx += w[tx] * ph[tx];
        acc.add(sx * w[PMAX + ty] * w[2 * PMAX + tz]);
      }
      acc.warp_reduce();
      if (lane == si) {
        ks = acc.s;
        kc = acc.c;
      }
    }
    if (lane < ns) {
      const int i = i0 + lane;
      const size_t k = (size_t)rep * ne + i;
      const double bi = -(KE * phi_real[k] + ((double)ks + (double)kc)) - slab_coef * ez[i] * scal[rep * NSCAL + S_QZ_ELYT];
      b[(size_t)rep * ldb + i] = bi;
      if (b32) {
        const float hi = (float)bi;
        b32[(size_t)rep * 2 * ldx + i] = hi;
        b32[(size_t)rep * 2 * ldx + ldx + i] = (float)(bi - (double)hi);
      }
    }
  }
}

// k-space force on the electrolyte sites (input order): F = -Q grad(phi_mesh) + Q E_z z-hat plus the
// real-space force f_pair, written (not added) at the site's index.  E_z = -dpsi / L_z (finite field) - KE 4 pi / V M_z (slab).
template <typename T>
__global__ void __launch_bounds__(256) k_gather_f_elyt(int nb, const T* __restrict__ phi, const int* __restrict__ off,
                                                       int cap, SpmeGeom sg,
                                                       const typename Vec4<T>::type* __restrict__ l_tmp,
                                                       const int* __restrict__ l_cell, const int* __restrict__ splI,
                                                       const T* __restrict__ splF, const double* __restrict__ dpsi,
                                                       double ff_over_lz, double slab_coef,
                                                       const double* __restrict__ scal,
                                                       const double* __restrict__ f_pair,
                                                       const float* __restrict__ f_sorted, double* __restrict__ F,
                                                       const int* __restrict__ srt) {
  pdl_enter();
  __shared__ T sw[8][kSiteBatch][3][PMAX], sdw[8][kSiteBatch][3][PMAX];
  __shared__ int si0[8][kSiteBatch][3];
  __shared__ T sq[8][kSiteBatch];
  const int rep = blockIdx.y;
  const int o = off[rep];
  const int n = min(off[rep + 1] - o, cap);
  const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5;
  const int P = sg.P, K1 = sg.K[0], K2 = sg.K[1], K3 = sg.K[2];
  const float inv_p = 1.0f / (float)P;
  // the lane's (y, z) stencil tasks (lane and lane + 32), computed once: the int <-> float
  // conversions of the row index stay out of the per-site loops
  const int ty0 = task_row(lane, inv_p), tz0 = lane - ty0 * P;
  const int ty1 = task_row(lane + 32, inv_p), tz1 = lane + 32 - ty1 * P;
  const T* m = phi + (size_t)rep * sg.Mr_s;
  const int nw = (gridDim.x * blockDim.x) >> 5;
  const int first = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const double mz = scal[rep * NSCAL + S_QZ_ELYT] + scal[rep * NSCAL + S_QZ_ELEC];
  const double ezf = -dpsi[rep] * ff_over_lz - slab_coef * mz;
  for (int i0 = first * nb; i0 < n; i0 += nw * nb) {
    batch_weights<T>(i0, n, nb, (size_t)rep * cap, l_tmp, l_cell, sg, splI, splF, lane, sw[wib], sdw[wib], si0[wib],
                     sq[wib], srt);
    const int cnt = min(nb, n - i0);
    T kx = 0, ky = 0, kz = 0;                  // lane si: site si's mesh gradient sums
    for (int si = 0; si < cnt; ++si) {
      const int* b0 = si0[wib][si];
      const T (*w)[PMAX] = sw[wib][si];
      const T (*dw)[PMAX] = sdw[wib][si];
      T gx = 0, gy = 0, gz = 0;
      for (int task = lane; task < P * P; task += 32) {
        const int ty = task < 32 ? ty0 : ty1, tz = task < 32 ? tz0 : tz1;
        const int jy = wrap_near(b0[1] - ty, K2), jz = wrap_near(b0[2] - tz, K3);
        // the P mesh loads of the x line issued together (unrolled to the largest order)
        T ph[PMAX];
#pragma unroll
        for (int tx = 0; tx < PMAX; ++tx)
          ph[tx] = tx < P ? m[((size_t)wrap_near(b0[0] - tx, K1) * K2 + jy) * K3 + jz] : T(0);
        T a = 0, ad = 0;
#pragma unroll
        for (int tx = 0; tx < PMAX; ++tx) {
          if (tx < P) {
            a += w[0][tx] * ph[tx];
            ad += dw[0][tx] * ph[tx];
          }
        }
        const T wy = w[1][ty], wz = w[2][tz];
        gx += ad * wy * wz;
        gy += a * dw[1][ty] * wz;
        gz += a * wy * dw[2][tz];
      }
      gx = warp_sum_t(gx);
      gy = warp_sum_t(gy);
      gz = warp_sum_t(gz);
      if (lane == si) {
        kx = gx;
        ky = gy;
        kz = gz;
      }
    }
    // the float64 epilogue once per batch, one lane per site (float64 instructions are costly on
    // GB300's narrow float64 pipe, so none is issued per site by a single lane)
    if (lane < cnt) {
      const int i = srt ? srt[(size_t)rep * cap + i0 + lane] : i0 + lane;      // input index
      const double q = (double)sq[wib][lane];
      const size_t gi = 3 * (size_t)(o + i);
      // the real-space force, by input index, or by sorted index (f_sorted, srt given)
      double fp[3] = {0.0, 0.0, 0.0};    // no real-space force: added later by k_add_pair_forces
      if (f_sorted) {
        const float* fs = f_sorted + 3 * ((size_t)rep * cap + i0 + lane);
        fp[0] = (double)fs[0];
        fp[1] = (double)fs[1];
        fp[2] = (double)fs[2];
      } else if (f_pair) {
        const double* fd = f_pair + 3 * ((size_t)rep * cap + i);
        fp[0] = fd[0];
        fp[1] = fd[1];
        fp[2] = fd[2];
      }
      F[gi + 0] = -q * (double)kx * sg.kl[0] + fp[0];
      F[gi + 1] = -q * (double)ky * sg.kl[1] + fp[1];
      F[gi + 2] = -q * (double)kz * sg.kl[2] + q * ezf + fp[2];
    }
    __syncwarp();
  }
}

// k-space force on electrode sites through the fixed stencils (written, not added).  A warp takes
// grp (1..32) consecutive sites: each site's stencil over the lanes, reduced in float32, lane s
// keeping site s's sums; the float64 epilogue then runs once per group, one lane per site.
// F += the real-space electrolyte forces, when the mesh part was gathered before the pair
// kernels finished: from f_pair (input order) or f_sorted (float32, cell-sorted order); one thread
// per sorted site, grid.y = replica.
__global__ void __launch_bounds__(256) k_add_pair_forces(const int* __restrict__ off, int cap,
                                                         const int* __restrict__ srt,
                                                         const double* __restrict__ f_pair,
                                                         const float* __restrict__ f_sorted, double* __restrict__ F) {
  pdl_enter();
  const int rep = blockIdx.y;
  const int o = off[rep];
  const int n = min(off[rep + 1] - o, cap);
  const int k = blockIdx.x * blockDim.x + threadIdx.x;
  if (k >= n) return;
  const int i = srt[(size_t)rep * cap + k];
  double* f = F + 3 * (size_t)(o + i);
  if (f_sorted) {
    const float* fs = f_sorted + 3 * ((size_t)rep * cap + k);
    f[0] += (double)fs[0];
    f[1] += (double)fs[1];
    f[2] += (double)fs[2];
  } else {
    const double* fd = f_pair + 3 * ((size_t)rep * cap + i);
    f[0] += fd[0];
    f[1] += fd[1];
    f[2] += fd[2];
  }
}

template <typename T>
__global__ void __launch_bounds__(256) k_gather_f_elec(const T* __restrict__ phi, const T* __restrict__ qT,
                                                       int ne, const int4* __restrict__ base,
                                                       const T* __restrict__ th, const T* __restrict__ dth,
                                                       SpmeGeom sg, const double* __restrict__ dpsi,
                                                       double ff_over_lz, double slab_coef,
                                                       const double* __restrict__ scal,
                                                       const double* __restrict__ efield, double* __restrict__ F,
                                                       int grp) {
  pdl_enter();
  const int rep = blockIdx.y;
  const int lane = threadIdx.x & 31;
  const int P = sg.P, K1 = sg.K[0], K2 = sg.K[1], K3 = sg.K[2];
  const float inv_p = 1.0f / (float)P;
  // the lane's (y, z) stencil tasks (lane and lane + 32), computed once: the int <-> float
  // conversions of the row index stay out of the per-site loops
  const int ty0 = task_row(lane, inv_p), tz0 = lane - ty0 * P;
  const int ty1 = task_row(lane + 32, inv_p), tz1 = lane + 32 - ty1 * P;
  const T* m = phi + (size_t)rep * sg.Mr_s;
  const int nwarp = (gridDim.x * blockDim.x) >> 5;
  for (int i0 = ((blockIdx.x * blockDim.x + threadIdx.x) >> 5) * grp; i0 < ne; i0 += nwarp * grp) {
    const int ns = min(grp, ne - i0);
    T kx = 0, ky = 0, kz = 0;
    for (int si = 0; si < ns; ++si) {
      const int i = i0 + si;
      const int4 bs = base[i];
      const T* w = th + (size_t)i * 3 * PMAX;
      const T* dw = dth + (size_t)i * 3 * PMAX;
      T gx = 0, gy = 0, gz = 0;
      for (int task = lane; task < P * P; task += 32) {
        const int ty = task < 32 ? ty0 : ty1, tz = task < 32 ? tz0 : tz1;
        const int jy = wrap_near(bs.y - ty, K2), jz = wrap_near(bs.z - tz, K3);
        T ph[PMAX];
#pragma unroll
        for (int tx = 0; tx < PMAX; ++tx)
          ph[tx] = tx < P ? m[((size_t)wrap_near(bs.x - tx, K1) * K2 + jy) * K3 + jz] : T(0);
        T a = 0, ad = 0;
#pragma unroll
        for (int tx = 0; tx < PMAX; ++tx) {
          if (tx < P) {
            a += w[tx] * ph[tx];
            ad += dw[tx] * ph[tx];
          }
        }
        const T wy = w[PMAX + ty], wz = w[2 * PMAX + tz];
        gx += ad * wy * wz;
        gy += a * dw[PMAX + ty] * wz;
        gz += a * wy * dw[2 * PMAX + tz];
      }
      gx = warp_sum_t(gx);
      gy = warp_sum_t(gy);
      gz = warp_sum_t(gz);
      if (lane == si) {
        kx = gx;
        ky = gy;
        kz = gz;
      }
    }
    if (lane < ns) {
      const int i = i0 + lane;
      const double qi = (double)qT[(size_t)rep * ne + i];
      const double mz = scal[rep * NSCAL + S_QZ_ELYT] + scal[rep * NSCAL + S_QZ_ELEC];
      const double ezf = -dpsi[rep] * ff_over_lz - slab_coef * mz;
      const size_t k = 3 * ((size_t)rep * ne + i);
      // + the electrolyte's real-space field at the site, when the b pass computed it
      const double rx = efield ? efield[k + 0] : 0.0, ry = efield ? efield[k + 1] : 0.0,
                   rz = efield ? efield[k + 2] : 0.0;
      F[k + 0] = qi * (rx - (double)kx * sg.kl[0]);
      F[k + 1] = qi * (ry - (double)ky * sg.kl[1]);
      F[k + 2] = qi * (rz - (double)kz * sg.kl[2] + ezf);
    }
  }
}

// ------------------------------------------------------------------------------------------
// S-apply: q_raw = S b + dpsi S v for R replicas per pass, one warp per row (rows grid-strided),
// S streamed once with 16-byte loads, several loads in flight per lane.
//   float32 S (mixed): b enters as the float32 split hi + lo, each 4-element group is summed in
//   float32 and the groups are added with TwoSum compensation, lanes combine (sum, error) pairs.
//   float64 S: float64 FMAs.
// The epilogue accumulates C^T q_raw and (A^-1 C)^T b for the projection.
// ------------------------------------------------------------------------------------------
template <int R>
__device__ __forceinline__ void sapply_epilogue(int i, int lane, int rep0, int nrep, int qstride, const double (&tot)[R],
                                                const double* __restrict__ b, int ldb, const double* __restrict__ dpsi,
                                                const double* __restrict__ Sv, const double* __restrict__ W,
                                                const double* __restrict__ c1, double* __restrict__ qout,
                                                double (&red)[4 * R]) {
  if (lane != 0) return;
  const double w0 = W[2 * i], w1 = W[2 * i + 1], cc = c1[i], svi = Sv[i];
#pragma unroll
  for (int r = 0; r < R; ++r) {
    const int rr = rep0 + r;
    if (rr >= nrep) break;
    const double qr = tot[r] + dpsi[rr] * svi;
    qout[(size_t)rr * qstride + i] = qr;
    const double bi = b[(size_t)rr * ldb + i];
    red[4 * r + 0] += qr;
    red[4 * r + 1] += qr * cc;
    red[4 * r + 2] += w0 * bi;
    red[4 * r + 3] += w1 * bi;
  }
}

template <int R>
__device__ __forceinline__ void sapply_reduce(const double (&red)[4 * R], int rep0, int nrep, double* scal) {
  __shared__ double sred[4 * R][8];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
  if (lane == 0)
    for (int k = 0; k < 4 * R; ++k) sred[k][warp] = red[k];
  __syncthreads();
  if (threadIdx.x < 4 * R) {
    const int k = threadIdx.x, r = k / 4, which = k % 4;
    if (rep0 + r < nrep) {
      double s = 0;
      for (int w = 0; w < nw; ++w) s += sred[k][w];
      atomicAdd(&scal[(rep0 + r) * NSCAL + S_CQ0 + which], s);
    }
  }
}

template <int R>
__global__ void __launch_bounds__(256) k_sapply32(const float* __restrict__ S, int ld, int ne,
                                                  const float* __restrict__ b32, int xstride, int xlo,
                                                  const double* __restrict__ b, int ldb, int rep0, int nrep,
                                                  const double* __restrict__ dpsi, const double* __restrict__ Sv,
                                                  const double* __restrict__ W, const double* __restrict__ c1,
                                                  double* __restrict__ qout, int qstride, double* __restrict__ scal) {
  pdl_enter();
  const int lane = threadIdx.x & 31;
  const int n4 = ld >> 2;
  double red[4 * R];
#pragma unroll
  for (int k = 0; k < 4 * R; ++k) red[k] = 0.0;
  const float4* yh[R];
  const float4* yl[R];
#pragma unroll
  for (int r = 0; r < R; ++r) {
    const int rr = min(rep0 + r, nrep - 1);
    yh[r] = reinterpret_cast<const float4*>(b32 + (size_t)rr * xstride);
    yl[r] = reinterpret_cast<const float4*>(b32 + (size_t)rr * xstride + xlo);
  }
  for (int i = (blockIdx.x * blockDim.x + threadIdx.x) >> 5; i < ne; i += (gridDim.x * blockDim.x) >> 5) {
    const float4* row = reinterpret_cast<const float4*>(S + (size_t)i * ld);
    Acc<float> acc[R];
    float lo[R];
#pragma unroll
    for (int r = 0; r < R; ++r) lo[r] = 0.f;
    constexpr int U = (R >= 4) ? 4 : 8;        // float4 loads of S in flight per lane
    for (int jb = lane; jb < n4; jb += 32 * U) {
      float4 sv[U];
#pragma unroll
      for (int u = 0; u < U; ++u) {
        const int j = jb + 32 * u;
        sv[u] = (j < n4) ? __ldcs(row + j) : make_float4(0.f, 0.f, 0.f, 0.f);
      }
#pragma unroll
      for (int u = 0; u < U; ++u) {
        const int j = min(jb + 32 * u, n4 - 1);    // out-of-range slots hold zeros in sv
#pragma unroll
        for (int r = 0; r < R; ++r) {
          const float4 h = yh[r][j], l = yl[r][j];
          acc[r].add(sv[u].x * h.x + sv[u].y * h.y + sv[u].z * h.z + sv[u].w * h.w);
          lo[r] += sv[u].x * l.x + sv[u].y * l.y + sv[u].z * l.z + sv[u].w * l.w;
        }
      }
    }
    double tot[R];
#pragma unroll
    for (int r = 0; r < R; ++r) {
      acc[r].add(lo[r]);
      acc[r].warp_reduce();
      tot[r] = acc[r].value();
    }
    sapply_epilogue<R>(i, lane, rep0, nrep, qstride, tot, b, ldb, dpsi, Sv, W, c1, qout, red);
  }
  sapply_reduce<R>(red, rep0, nrep, scal);
}

template <int R>
__global__ void __launch_bounds__(256) k_sapply64(const double* __restrict__ S, int ld, int ne,
                                                  const double* __restrict__ b, int ldb, int rep0, int nrep,
                                                  const double* __restrict__ dpsi, const double* __restrict__ Sv,
                                                  const double* __restrict__ W, const double* __restrict__ c1,
                                                  double* __restrict__ qout, int qstride, double* __restrict__ scal) {
  pdl_enter();
  const int lane = threadIdx.x & 31;
  double red[4 * R];
#pragma unroll
  for (int k = 0; k < 4 * R; ++k) red[k] = 0.0;
  for (int i = (blockIdx.x * blockDim.x + threadIdx.x) >> 5; i < ne; i += (gridDim.x * blockDim.x) >> 5) {
    // rows and b are padded to ld (a multiple of 4) with zeros, so whole double2 pairs are read
    const double2* row = reinterpret_cast<const double2*>(S + (size_t)i * ld);
    double acc[R];
#pragma unroll
    for (int r = 0; r < R; ++r) acc[r] = 0.0;
    const int n2 = ld >> 1;
#pragma unroll 4
    for (int j = lane; j < n2; j += 32) {
      const double2 sv = __ldcs(row + j);
#pragma unroll
      for (int r = 0; r < R; ++r) {
        const int rr = min(rep0 + r, nrep - 1);
        const double2 y = reinterpret_cast<const double2*>(b + (size_t)rr * ldb)[j];
        acc[r] = fma(sv.x, y.x, fma(sv.y, y.y, acc[r]));
      }
    }
    double tot[R];
#pragma unroll
    for (int r = 0; r < R; ++r) tot[r] = warp_sum(acc[r]);
    sapply_epilogue<R>(i, lane, rep0, nrep, qstride, tot, b, ldb, dpsi, Sv, W, c1, qout, red);
  }
  sapply_reduce<R>(red, rep0, nrep, scal);
}

// ------------------------------------------------------------------------------------------
// Streaming S-apply (mixed precision, one replica): persistent CTAs, one per SM, each holding the
// whole right-hand side (float32 hi and lo halves, 8 ld bytes) in shared memory.  The flattened S
// (rows x ld/4 float4, contiguous) is cut into one equal contiguous span per warp, so every warp
// streams the same number of bytes whatever the row count; a span covers whole and partial rows,
// and each row segment's compensated dot product is added into qpart[row] in float64 (at most a
// few segments per row).  k_sapply_finish then forms q_raw = qpart + dpsi S v with the projection
// sums and clears qpart for the next call.
// ------------------------------------------------------------------------------------------
constexpr int SS_THREADS = 512;
constexpr int SS_SMEM_MAX = 200 * 1024;      // largest staged right-hand side (bytes)

template <int U>
__global__ void __launch_bounds__(SS_THREADS, 1) k_sapply_stream(const float* __restrict__ S, int ld, int rows,
                                                                 const float* __restrict__ xh,
                                                                 const float* __restrict__ xl,
                                                                 double* __restrict__ qpart) {
  pdl_enter();
  extern __shared__ float4 ss_x[];
  const int n4 = ld >> 2;
  float4* shi = ss_x;
  float4* slo = ss_x + n4;
  const float4* gh = reinterpret_cast<const float4*>(xh);
  const float4* gl = reinterpret_cast<const float4*>(xl);
  for (int k = threadIdx.x; k < n4; k += blockDim.x) {
    shi[k] = gh[k];
    slo[k] = gl[k];
  }
  __syncthreads();
  const int lane = threadIdx.x & 31;
  const long long nw = (long long)gridDim.x * (blockDim.x >> 5);
  const long long wid = (long long)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
  const long long total = (long long)rows * n4;
  const long long per = (total + nw - 1) / nw;
  long long p = wid * per;
  const long long pend = min(total, p + per);
  const float4* S4 = reinterpret_cast<const float4*>(S);
  while (p < pend) {
    const int row = (int)(p / n4);
    const long long rbase = (long long)row * n4;
    const int c0 = (int)(p - rbase);
    const int c1 = (int)(min(pend, rbase + n4) - rbase);
    const float4* srow = S4 + rbase;
    Acc<float> acc;
    float lo = 0.f;
    for (int jb = c0 + lane; jb < c1; jb += 32 * U) {
      float4 sv[U];
#pragma unroll
      for (int u = 0; u < U; ++u) {
        const int j = jb + 32 * u;
        sv[u] = (j < c1) ? __ldcs(srow + j) : make_float4(0.f, 0.f, 0.f, 0.f);
      }
#pragma unroll
      for (int u = 0; u < U; ++u) {
        const int j = min(jb + 32 * u, c1 - 1);    // out-of-range slots hold zeros in sv
        const float4 h = shi[j], l = slo[j];
        acc.add(sv[u].x * h.x + sv[u].y * h.y + sv[u].z * h.z + sv[u].w * h.w);
        lo += sv[u].x * l.x + sv[u].y * l.y + sv[u].z * l.z + sv[u].w * l.w;
      }
    }
    acc.add(lo);
    acc.warp_reduce();
    if (lane == 0) atomicAdd(&qpart[row], acc.value());
    p = rbase + c1;
  }
}

// q_raw = qpart + dpsi S v (one replica), qpart cleared; the projection sums C^T q_raw and
// (A^-1 C)^T b as in the S-apply epilogue.
__global__ void __launch_bounds__(FIN_THREADS) k_sapply_finish(int rows, double* __restrict__ qpart,
                                                       const double* __restrict__ b, const double* __restrict__ dpsi,
                                                       const double* __restrict__ Sv, const double* __restrict__ W,
                                                       const double* __restrict__ c1, double* __restrict__ qout,
                                                       double* __restrict__ scal) {
  pdl_enter();
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  double red[4] = {0, 0, 0, 0};
  if (i < rows) {
    const double qr = qpart[i] + dpsi[0] * Sv[i];
    qpart[i] = 0.0;
    qout[i] = qr;
    const double bi = b[i];
    red[0] = qr;
    red[1] = qr * c1[i];
    red[2] = W[2 * i] * bi;
    red[3] = W[2 * i + 1] * bi;
  }
#pragma unroll
  for (int k = 0; k < 4; ++k) red[k] = warp_sum(red[k]);
  double* const dst[4] = {scal + S_CQ0, scal + S_CQ1, scal + S_WB0, scal + S_WB1};
  block_atomic_add<4>(red, dst);
}

// ------------------------------------------------------------------------------------------
// Batched S-apply on the 5th-generation tensor cores: D = S Y^T for up to 256 replicas per pass,
// Y the replicas' right-hand sides.  tcgen05.mma kind::tf32, M = 128 rows of S per CTA, N = the
// replica tile, K = 8 per instruction, accumulator in TMEM.  Split-TF32 ("3xTF32"): with
// x_hi = x with its low 13 mantissa bits cleared and x_lo = x - x_hi,
//   S Y ~= S_hi Y_hi + S_hi Y_lo + S_lo Y_hi   (the dropped S_lo Y_lo term is ~2^-22 relative),
// accumulated in float32.  Operands are staged into shared memory in the canonical K-major,
// no-swizzle layout: 8-row x 16-byte core matrices, K-direction core-matrix stride LBO = 128 B,
// 8-row-group stride SBO = 1024 B for a 32-element K chunk.  Split-K across CTAs; partial tiles
// are added into D with float32 atomics (D cleared by the host first).
// ------------------------------------------------------------------------------------------
constexpr int TC_M = 128, TC_KC = 32, TC_THREADS = 128;
constexpr int TC_MIN_REPLICAS = 8;     // batches this large take the tensor-core path (mixed precision)

__device__ __forceinline__ uint32_t smem_u32(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }

__device__ __forceinline__ uint64_t umma_desc(uint32_t saddr, uint32_t lbo, uint32_t sbo) {
  uint64_t d = (uint64_t)((saddr & 0x3FFFF) >> 4);
  d |= (uint64_t)((lbo >> 4) & 0x3FFF) << 16;
  d |= (uint64_t)((sbo >> 4) & 0x3FFF) << 32;
  d |= (uint64_t)1 << 46;                      // descriptor version of sm_100-class tensor cores
  return d;                                    // base offset 0, no swizzle
}

__device__ __forceinline__ float tf32_hi(float x) { return __uint_as_float(__float_as_uint(x) & 0xFFFFE000u); }

// byte offset of element (row, k) of a K-major operand chunk with TC_KC columns
__device__ __forceinline__ int tc_off(int row, int k4) { return ((row >> 3) * (TC_KC / 4) + k4) * 128 + (row & 7) * 16; }

template <int NT>
__global__ void __launch_bounds__(TC_THREADS) k_sapply_tc(const float* __restrict__ S, int ld, int ne,
                                                          const float* __restrict__ b32, int rep0, int nrep,
                                                          int chunks_per_split, float* __restrict__ D,
                                                          int short_wait, int* __restrict__ status) {
  static_assert(NT % 16 == 0 && NT >= 16 && NT <= 256, "replica tile");
  constexpr int TMEM_COLS = NT < 32 ? 32 : NT;
  constexpr int A_BYTES = TC_M * TC_KC * 4, B_BYTES = NT * TC_KC * 4;
  extern __shared__ __align__(1024) unsigned char tsm[];
  unsigned char* sAh = tsm;
  unsigned char* sAl = tsm + A_BYTES;
  unsigned char* sBh = tsm + 2 * A_BYTES;
  unsigned char* sBl = tsm + 2 * A_BYTES + B_BYTES;
  __shared__ __align__(8) uint64_t mbar;
  __shared__ uint32_t tslot;
  __shared__ int s_abort;
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int m0 = blockIdx.x * TC_M;
  const int nchunks = (ld + TC_KC - 1) / TC_KC;
  const int c_begin = blockIdx.y * chunks_per_split, c_end = min(nchunks, c_begin + chunks_per_split);
  if (c_begin >= c_end) return;

  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(&tslot)),
                 "r"(TMEM_COLS));
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
  }
  if (tid == 0) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(&mbar)), "r"(1));
    asm volatile("fence.mbarrier_init.release.cluster;");
    s_abort = 0;
  }
  asm volatile("tcgen05.fence::before_thread_sync;");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;");
  const uint32_t taddr = tslot;
  const uint32_t idesc = (1u << 4) | (2u << 7) | (2u << 10) | ((uint32_t)(NT >> 3) << 17) | ((uint32_t)(TC_M >> 4) << 24);
  const int ld4 = ld >> 2;
  int phase = 0;
  bool ok = true;

  for (int ch = c_begin; ch < c_end && ok; ++ch) {
    const int k40 = ch * (TC_KC / 4);          // first float4 column of the chunk
    // ---- stage S rows m0 .. m0+127 (thread = row), split into tf32 hi / lo
    {
      const int m = m0 + tid;
      const float4* row = reinterpret_cast<const float4*>(S + (size_t)min(m, ne - 1) * ld);
#pragma unroll
      for (int j = 0; j < TC_KC / 4; ++j) {
        float4 v = make_float4(0.f, 0.f, 0.f, 0.f);
        if (m < ne && k40 + j < ld4) v = __ldg(row + k40 + j);
        const float4 h = make_float4(tf32_hi(v.x), tf32_hi(v.y), tf32_hi(v.z), tf32_hi(v.w));
        const float4 l = make_float4(v.x - h.x, v.y - h.y, v.z - h.z, v.w - h.w);
        *reinterpret_cast<float4*>(sAh + tc_off(tid, j)) = h;
        *reinterpret_cast<float4*>(sAl + tc_off(tid, j)) = l;
      }
    }
    // ---- stage Y rows (replicas) rep0 .. rep0+NT-1: y = hi32 + lo32 -> tf32 hi / lo
    for (int n = tid; n < NT; n += TC_THREADS) {
      const bool live = rep0 + n < nrep;
      const float4* yh = reinterpret_cast<const float4*>(b32 + (size_t)min(rep0 + n, nrep - 1) * 2 * ld);
      const float4* yl = reinterpret_cast<const float4*>(b32 + (size_t)min(rep0 + n, nrep - 1) * 2 * ld + ld);
#pragma unroll
      for (int j = 0; j < TC_KC / 4; ++j) {
        float4 a = make_float4(0.f, 0.f, 0.f, 0.f), c = a;
        if (live && k40 + j < ld4) {
          a = yh[k40 + j];
          c = yl[k40 + j];
        }
        const float4 h = make_float4(tf32_hi(a.x), tf32_hi(a.y), tf32_hi(a.z), tf32_hi(a.w));
        const float4 l = make_float4((a.x - h.x) + c.x, (a.y - h.y) + c.y, (a.z - h.z) + c.z, (a.w - h.w) + c.w);
        *reinterpret_cast<float4*>(sBh + tc_off(n, j)) = h;
        *reinterpret_cast<float4*>(sBl + tc_off(n, j)) = l;
      }
    }
    asm volatile("fence.proxy.async.shared::cta;");     // make the staged operands visible to the tensor cores
    asm volatile("tcgen05.fence::before_thread_sync;");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;");
    if (tid == 0) {
#pragma unroll
      for (int kk = 0; kk < TC_KC / 8; ++kk) {
        const uint32_t koff = kk * 256;                  // two core matrices along K per instruction
        const uint64_t ah = umma_desc(smem_u32(sAh) + koff, 128, 1024);
        const uint64_t al = umma_desc(smem_u32(sAl) + koff, 128, 1024);
        const uint64_t bh = umma_desc(smem_u32(sBh) + koff, 128, 1024);
        const uint64_t bl = umma_desc(smem_u32(sBl) + koff, 128, 1024);
        const uint32_t acc0 = (ch > c_begin || kk > 0) ? 1u : 0u;
        asm volatile("{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n}" ::"r"(taddr),
                     "l"(ah), "l"(bh), "r"(idesc), "r"(acc0));
        asm volatile("{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n}" ::"r"(taddr),
                     "l"(ah), "l"(bl), "r"(idesc), "r"(1u));
        asm volatile("{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n}" ::"r"(taddr),
                     "l"(al), "l"(bh), "r"(idesc), "r"(1u));
      }
      asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(smem_u32(&mbar)));
    }
    // ---- bounded wait for the MMAs (they read the staged operands, so no restaging before);
    // short_wait (cpm_set_wait_test) makes it give up without polling
    bool done = false;
    const int first_limit = short_wait ? 0 : (1 << 22);
    for (int it = 0; it < first_limit && !done; ++it) {
      uint32_t r;
      asm volatile("{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}"
                   : "=r"(r) : "r"(smem_u32(&mbar)), "r"(phase) : "memory");
      done = r != 0;
      if (!done) __nanosleep(32);
    }
    if (!done) {
      s_abort = 1;
      // a second bounded wait for MMAs still in flight: they read the staged operands and write
      // the TMEM accumulator that is freed below
      for (int it = 0; it < (1 << 22) && !done; ++it) {
        uint32_t r;
        asm volatile("{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}"
                     : "=r"(r) : "r"(smem_u32(&mbar)), "r"(phase) : "memory");
        done = r != 0;
        if (!done) __nanosleep(32);
      }
    }
    phase ^= 1;
    __syncthreads();
    ok = (s_abort == 0);
  }
  asm volatile("tcgen05.fence::after_thread_sync;");
  if (ok) {
    const int m = m0 + warp * 32 + lane;
#pragma unroll
    for (int n0 = 0; n0 < NT; n0 += 16) {
      uint32_t r[16];
      asm volatile("tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];"
                   : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
                     "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
                   : "r"(taddr + ((uint32_t)(warp * 32) << 16) + (uint32_t)n0));
      asm volatile("tcgen05.wait::ld.sync.aligned;");
      if (m < ne) {
#pragma unroll
        for (int j = 0; j < 16; ++j) {
          const int rep = rep0 + n0 + j;
          if (rep < nrep) atomicAdd(&D[(size_t)rep * ne + m], __uint_as_float(r[j]));
        }
      }
    }
  } else if (tid == 0) {
    latch_error(status, DE_TIMEOUT);
  }
  asm volatile("tcgen05.fence::before_thread_sync;");
  __syncthreads();
  if (warp == 0) asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(taddr), "r"(TMEM_COLS));
}

// q_raw = D + dpsi S v in float64 per (replica, site), with the projection sums C^T q_raw and
// (A^-1 C)^T b; one thread per site, grid.y = replica.
__global__ void __launch_bounds__(256) k_qraw_epilogue(const float* __restrict__ D, int ne, const double* __restrict__ b,
                                                       int ldb, const double* __restrict__ dpsi,
                                                       const double* __restrict__ Sv, const double* __restrict__ W,
                                                       const double* __restrict__ c1, double* __restrict__ q,
                                                       double* __restrict__ scal) {
  pdl_enter();
  const int rep = blockIdx.y;
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  double red[4] = {0, 0, 0, 0};
  if (i < ne) {
    const double qr = (double)D[(size_t)rep * ne + i] + dpsi[rep] * Sv[i];
    q[(size_t)rep * ne + i] = qr;
    const double bi = b[(size_t)rep * ldb + i];
    red[0] = qr;
    red[1] = qr * c1[i];
    red[2] = W[2 * i] * bi;
    red[3] = W[2 * i + 1] * bi;
  }
#pragma unroll
  for (int k = 0; k < 4; ++k) red[k] = warp_sum(red[k]);
  double* const dst[4] = {scal + rep * NSCAL + S_CQ0, scal + rep * NSCAL + S_CQ1, scal + rep * NSCAL + S_WB0,
                          scal + rep * NSCAL + S_WB1};
  block_atomic_add<4>(red, dst);
}

// q = q_raw - A^-1 C M C^T q_raw (restores C^T q = 0 to float64 rounding); psibar = -M (A^-1 C)^T (b + dpsi v).
// Also accumulates q^T b for the closed-form energy.
// The force pass's view of the final charges, produced by the projection of the same call (the
// work of k_charge_prep, without its own launch): q in the working precision and the float64
// sums q z, q v, q^2, q_+.
template <typename T> struct ChargePrep {
  T* qT;                       // [nrep][ne]
  const double* ez;
  const double* ev;
  const double* eplus;
};

template <typename T>
__device__ __forceinline__ void prep_site(const ChargePrep<T>& cp, int rep, int ne, int i, double qi,
                                          double (&acc)[5]) {
  if (!cp.qT) return;                    // no force pass follows in this call
  cp.qT[(size_t)rep * ne + i] = (T)qi;
  acc[1] += qi * cp.ez[i];
  acc[2] += qi * cp.ev[i];
  acc[3] += qi * qi;
  acc[4] += qi * cp.eplus[i];
}

template <typename T>
__device__ __forceinline__ void project_sums(double (&acc)[5], double* s) {
#pragma unroll
  for (int k = 0; k < 5; ++k) acc[k] = warp_sum(acc[k]);
  double* const dst[5] = {s + S_QB, s + S_QZ_ELEC, s + S_QV_ELEC, s + S_QQ_ELEC, s + S_QPLUS};
  block_atomic_add<5>(acc, dst);
}

// q_raw held as the packed S-apply's row accumulator (one replica): q_raw = part + dpsi S v, and
// the projection clears part for the next call; the S-apply's sums S_CQ0, S_CQ1 leave out the
// dpsi S v terms, dpsi (sv0, sv1) = dpsi (1^T S v, c1^T S v).  part == nullptr: q_raw is in the
// charge array and the sums are complete.
struct QRawPart {
  double* part;
  const double* Sv;
  double sv0, sv1;
};

__device__ __forceinline__ double qraw_take(const QRawPart& qp, int i, double dpsi) {
  const double r = qp.part[i] + dpsi * qp.Sv[i];
  qp.part[i] = 0.0;
  return r;
}

template <typename T>
__global__ void __launch_bounds__(FIN_THREADS) k_project(double* __restrict__ q, int ne, int nrep, int ncons,
                                                 const double* __restrict__ W, const double* __restrict__ b, int ldb,
                                                 double* __restrict__ scal, const double* __restrict__ dpsi,
                                                 double m00, double m01, double m10, double m11, double wtv0,
                                                 double wtv1, double* __restrict__ psibar, ChargePrep<T> cp,
                                                 QRawPart qp) {
  pdl_enter();
  const int rep = blockIdx.y;
  double* s = scal + rep * NSCAL;
  const double dq0 = qp.part ? dpsi[rep] * qp.sv0 : 0.0, dq1 = qp.part ? dpsi[rep] * qp.sv1 : 0.0;
  const double c0 = s[S_CQ0] + dq0, cq1 = (ncons == 2) ? s[S_CQ1] + dq1 : 0.0;
  const double a0 = m00 * c0 + m01 * cq1, a1 = m10 * c0 + m11 * cq1;
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  double acc[5] = {0.0, 0.0, 0.0, 0.0, 0.0};
  if (i < ne) {
    double corr = W[2 * i] * a0;
    if (ncons == 2) corr += W[2 * i + 1] * a1;
    const size_t k = (size_t)rep * ne + i;
    const double qi = (qp.part ? qraw_take(qp, i, dpsi[rep]) : q[k]) - corr;
    q[k] = qi;
    acc[0] = qi * b[(size_t)rep * ldb + i];
    prep_site(cp, rep, ne, i, qi, acc);
  }
  if (i == 0 && psibar) {
    const double y0 = s[S_WB0] + dpsi[rep] * wtv0, y1 = (ncons == 2) ? s[S_WB1] + dpsi[rep] * wtv1 : 0.0;
    psibar[rep * ncons + 0] = -(m00 * y0 + m01 * y1);
    if (ncons == 2) psibar[rep * ncons + 1] = -(m10 * y0 + m11 * y1);
  }
  project_sums<T>(acc, s);
}

// Mirror form, before the S-apply: y+- = b_I0 +- b_J per mirror pair (float64, rows of length
// 2 ldh: y+ at [0, nh), y- at [ldh, ldh + nh)); with x32 != nullptr also the float32 hi / lo split,
// halves of length ldx = 2 ldh.  (The dpsi v part enters through S v.)
__global__ void __launch_bounds__(256) k_mirror_fold(const double* __restrict__ b, int ldb, int nh, int ldh,
                                                     const int* __restrict__ i0, const int* __restrict__ jm,
                                                     double* __restrict__ y, float* __restrict__ x32) {
  pdl_enter();
  const int rep = blockIdx.y;
  const int k = blockIdx.x * blockDim.x + threadIdx.x;
  if (k >= nh) return;
  const double bi = b[(size_t)rep * ldb + i0[k]], bj = b[(size_t)rep * ldb + jm[k]];
  const double yp = bi + bj, ym = bi - bj;
  double* yr = y + (size_t)rep * 2 * ldh;
  yr[k] = yp;
  yr[ldh + k] = ym;
  if (x32) {
    float* xr = x32 + (size_t)rep * 4 * ldh;
    const float hp = (float)yp, hm = (float)ym;
    xr[k] = hp;
    xr[ldh + k] = hm;
    xr[2 * ldh + k] = (float)(yp - (double)hp);
    xr[3 * ldh + k] = (float)(ym - (double)hm);
  }
}

// Mirror form, after the S-apply: q+- <- q+- - w+- M+- 1^T q+- (the S-apply accumulated
// S_CQ0 = 1^T q+ + 1^T q- and S_CQ1 = 1^T q-), then q_I0 = (q+ + q-) / 2, q_J = (q+ - q-) / 2.
// Offsets: with mu+- = -M+- w+-^T (y+- + dpsi v+-) (A+- q+- = y+- + dpsi v+- + mu+- 1), the full
// problem's A q = b + dpsi v + psibar e + psibar_1 e_1 gives psibar = (mu+ + mu-) / 2, psibar_1 = -mu-.
// Also accumulates q^T b for the closed-form energy.
template <typename T>
__global__ void __launch_bounds__(FIN_THREADS) k_project_mirror(const double* __restrict__ qpm, int nh,
                                                        const int* __restrict__ i0, const int* __restrict__ jm,
                                                        const double* __restrict__ W, const double* __restrict__ b,
                                                        int ldb, int ne, double* __restrict__ scal,
                                                        const double* __restrict__ dpsi, double mp, double mm,
                                                        double wtvp, double wtvm, double* __restrict__ q,
                                                        double* __restrict__ psibar, ChargePrep<T> cp, QRawPart qp) {
  pdl_enter();
  const int rep = blockIdx.y;
  double* s = scal + rep * NSCAL;
  const double dq0 = qp.part ? dpsi[rep] * qp.sv0 : 0.0, dq1 = qp.part ? dpsi[rep] * qp.sv1 : 0.0;
  const double cpl = (s[S_CQ0] + dq0) - (s[S_CQ1] + dq1), cm = s[S_CQ1] + dq1;
  const int k = blockIdx.x * blockDim.x + threadIdx.x;
  double acc[5] = {0.0, 0.0, 0.0, 0.0, 0.0};
  if (k < nh) {
    const double rp = qp.part ? qraw_take(qp, k, dpsi[rep]) : qpm[(size_t)rep * 2 * nh + k];
    const double rm = qp.part ? qraw_take(qp, nh + k, dpsi[rep]) : qpm[(size_t)rep * 2 * nh + nh + k];
    const double qpl = rp - W[2 * k] * mp * cpl;
    const double qm = rm - W[2 * (size_t)nh + 2 * k + 1] * mm * cm;
    const int i = i0[k], j = jm[k];
    const double qi = 0.5 * (qpl + qm), qj = 0.5 * (qpl - qm);
    q[(size_t)rep * ne + i] = qi;
    q[(size_t)rep * ne + j] = qj;
    acc[0] = qi * b[(size_t)rep * ldb + i] + qj * b[(size_t)rep * ldb + j];
    prep_site(cp, rep, ne, i, qi, acc);
    prep_site(cp, rep, ne, j, qj, acc);
  }
  if (k == 0 && psibar) {
    const double mup = -mp * (s[S_WB0] + dpsi[rep] * wtvp), mum = -mm * (s[S_WB1] + dpsi[rep] * wtvm);
    psibar[rep * 2 + 0] = 0.5 * (mup + mum);
    psibar[rep * 2 + 1] = -mum;
  }
  project_sums<T>(acc, s);
}

// Per replica (U, H, dH/d(dpsi), Q_+).  closed_form: at the constrained optimum Eq. 3 reduces to
// U = U_elyt - 1/2 q^T b + 1/2 dpsi q^T v (A q = b + dpsi v + C lam and C^T q = 0); otherwise U is the
// full Ewald sum of all charges (real space + mesh + self terms).
__global__ void k_energy_final(int nrep, const double* __restrict__ scal, const double* __restrict__ dpsi,
                               double alpha, double eta, double slab_e_coef, double ff_over_lz, int closed_form,
                               double* __restrict__ energy) {
  pdl_enter();
  const int rep = blockIdx.x * blockDim.x + threadIdx.x;
  if (rep >= nrep) return;
  const double* s = scal + rep * NSCAL;
  const double self_pt = alpha / sqrt(PI);
  double U;
  if (closed_form) {
    U = KE * (0.5 * s[S_E_LL] - self_pt * s[S_QQ_ELYT]) + s[S_E_RECIP_L] +
        slab_e_coef * s[S_QZ_ELYT] * s[S_QZ_ELYT] - 0.5 * s[S_QB] + 0.5 * dpsi[rep] * s[S_QV_ELEC];
  } else {
    U = KE * (0.5 * s[S_E_LL] + s[S_E_LE] + 0.5 * s[S_E_EE]) + s[S_E_RECIP] +
        KE * (-self_pt * (s[S_QQ_ELYT] + s[S_QQ_ELEC]) + eta / sqrt(2.0 * PI) * s[S_QQ_ELEC]);
    const double mz = s[S_QZ_ELYT] + s[S_QZ_ELEC];
    U += slab_e_coef * mz * mz;
  }
  const double dHdpsi = -s[S_QV_ELEC] + ff_over_lz * s[S_QZ_ELYT];
  energy[NENERGY * rep + 0] = U;
  energy[NENERGY * rep + 1] = U + dpsi[rep] * dHdpsi;
  energy[NENERGY * rep + 2] = dHdpsi;
  energy[NENERGY * rep + 3] = s[S_QPLUS];
}

// ------------------------------------------------------------------------------------------
// host orchestration
// ------------------------------------------------------------------------------------------
static CellGeom cell_geom(const cpm_ctx* c) {
  CellGeom g;
  g.nsten = 1;
  for (int d = 0; d < 3; ++d) {
    g.nc[d] = c->nc[d];
    g.sten[d] = c->sten[d];
    g.w[d] = 2 * c->sten[d] + 1;
    g.nsten *= g.w[d];
    g.edge[d] = c->edge[d];
    g.inv_edge[d] = 1.0 / c->edge[d];
    g.box[d] = c->ebox[d];
    g.inv_box[d] = 1.0 / c->ebox[d];
  }
  g.rc2 = c->p.rcut * c->p.rcut;
  g.alpha_f = (float)c->p.alpha;
  g.rc2_f = (float)g.rc2;
  for (int d = 0; d < 3; ++d) g.edge_f[d] = (float)g.edge[d];
  g.gz = c->pair_gz;
  g.ngz = (g.nc[2] + g.gz - 1) / g.gz;
  return g;
}

// Blocks of a pair-kernel launch per replica: one per (x, y) column and group of gz cells in z.
static int pair_blocks(const CellGeom& g) { return g.nc[0] * g.nc[1] * g.ngz; }

static SpmeGeom spme_geom(const cpm_ctx* c) {
  SpmeGeom s;
  for (int d = 0; d < 3; ++d) {
    s.K[d] = c->K[d];
    s.box[d] = c->ebox[d];
    s.kl[d] = c->K[d] / c->ebox[d];
  }
  s.spl_off[0] = 0;
  s.spl_off[1] = c->nc[0];
  s.spl_off[2] = c->nc[0] + c->nc[1];
  for (int d = 0; d < 3; ++d) s.nc[d] = c->nc[d];
  s.P = c->P;
  s.Mr_s = c->Mr_s;
  s.Mc_s = c->Mc_s;
  return s;
}

// Every kernel launch of a per-step call is counted (cpm_counters) and checked.
#define STEP_LAUNCH()  \
  do {                 \
    ++c->launches;     \
    CPM_LAUNCH();      \
  } while (0)

// Records a (start, stop) event pair around one phase when the profiler is on.
struct PhaseTimer {
  cpm_ctx* c;
  cudaStream_t st;
  int slot = -1;
  PhaseTimer(cpm_ctx* c_, cudaStream_t st_, int phase) : c(c_), st(st_) {
    if (c->prof_cap > 0 && c->prof_used < c->prof_cap) {
      slot = c->prof_used++;
      c->prof_phase[slot] = phase;
      cudaEventRecord(c->prof_ev[2 * slot], st);
    }
  }
  void stop() {
    if (slot >= 0) cudaEventRecord(c->prof_ev[2 * slot + 1], st);
    slot = -1;
  }
  ~PhaseTimer() { stop(); }
};

// Electrolyte sites per warp-batch of the mesh kernels: one while the sites leave SMs idle, up to
// kSiteBatch once every SM has about that many sites per resident warp.
static int site_batch(const cpm_ctx* c, int cap, int nrep) {
  const long long sites = (long long)cap * nrep;
  const long long warps = (long long)std::max(1, c->n_sm) * 32;
  return (int)std::max(1LL, std::min<long long>(kSiteBatch, sites / warps));
}

// Electrode sites (or pair-list rows) per warp in the electrode gathers and k_ee_forces: as many
// as keep about 32 warps per SM busy, at most 8 -- the float64 epilogue of a group runs once, one
// lane per site (float64 instructions are costly on GB300's narrow float64 pipe), while small
// electrodes keep one site per warp for parallelism.
static int elec_group(const cpm_ctx* c, int ne, int nrep) {
  const long long warps = (long long)std::max(1, c->n_sm) * 32;
  return (int)std::max(1LL, std::min<long long>(8, (long long)ne * nrep / warps));
}

static int grid_for(long long warps_needed, int per_block_warps = 8, int max_blocks = 152 * 16) {
  long long b = (warps_needed + per_block_warps - 1) / per_block_warps;
  return (int)std::max(1LL, std::min<long long>(b, max_blocks));
}

template <typename T> struct FftOps;
template <> struct FftOps<float> {
  static cufftResult fwd(cufftHandle h, void* in, void* out) { return cufftExecR2C(h, (cufftReal*)in, (cufftComplex*)out); }
  static cufftResult inv(cufftHandle h, void* in, void* out) { return cufftExecC2R(h, (cufftComplex*)in, (cufftReal*)out); }
  using C2 = float2;
};
template <> struct FftOps<double> {
  static cufftResult fwd(cufftHandle h, void* in, void* out) {
    return cufftExecD2Z(h, (cufftDoubleReal*)in, (cufftDoubleComplex*)out);
  }
  static cufftResult inv(cufftHandle h, void* in, void* out) {
    return cufftExecZ2D(h, (cufftDoubleComplex*)in, (cufftDoubleReal*)out);
  }
  using C2 = double2;
};

// mesh -> spectrum, influence (+ energy), spectrum -> potential mesh
template <typename T>
static int convolve(cpm_ctx* c, int nrep, int energy_slot, cudaStream_t st) {
  using C2 = typename FftOps<T>::C2;
  if (sizeof(T) == sizeof(float) && c->fft_variant == CPM_FFT_OWN && c->fft_own_ok)
    return cpm_internal_convolve_own(c, nrep, energy_slot, st);
  const int b = (nrep == c->p.max_replicas && c->have_plan[1]) ? 1 : 0;
  CPM_LIB(cufftSetStream(c->plan_r2c[b], st) == CUFFT_SUCCESS, "cufftSetStream");
  CPM_LIB(cufftSetStream(c->plan_c2r[b], st) == CUFFT_SUCCESS, "cufftSetStream");
  T* mr = (T*)c->mesh_r;
  C2* mc = (C2*)c->mesh_c;
  T* mp = (T*)c->mesh_phi;
  const int nexec = b ? 1 : nrep;
  for (int r = 0; r < nexec; ++r)
    CPM_LIB(FftOps<T>::fwd(c->plan_r2c[b], mr + r * c->Mr_s, mc + r * c->Mc_s) == CUFFT_SUCCESS, "cufftExec(r2c)");
  const T* G = c->mixed ? (const T*)c->G32 : (const T*)c->G64;
  const int blocks = (int)std::min<long long>((c->Mc + 255) / 256, 152 * 8);
  CPM_CUDA(launch_pdl(k_influence<T, C2>, dim3(blocks, nrep), 256, 0, st, mc, G, c->Mc, c->Mc_s, c->K[2] / 2 + 1, c->K[2],
                                                         energy_slot, c->scal));
  STEP_LAUNCH();
  for (int r = 0; r < nexec; ++r)
    CPM_LIB(FftOps<T>::inv(c->plan_c2r[b], mc + r * c->Mc_s, mp + r * c->Mr_s) == CUFFT_SUCCESS, "cufftExec(c2r)");
  return CPM_OK;
}

template <int NT>
static size_t tc_smem_bytes() {
  return 2 * (size_t)TC_M * TC_KC * 4 + 2 * (size_t)NT * TC_KC * 4;
}

template <int NT>
static int launch_tc(cpm_ctx* c, int rep0, int nrep, dim3 grid, int cps, cudaStream_t st) {
  k_sapply_tc<NT><<<grid, TC_THREADS, tc_smem_bytes<NT>(), st>>>(c->S32, c->ld32, c->ne, c->b32, rep0, nrep, cps,
                                                                  c->qraw32, c->wait_test ? 1 : 0, c->status);
  STEP_LAUNCH();
  return CPM_OK;
}

// D = S Y^T on the tensor cores for all replicas, in passes of at most 256; split-K so that the
// grid covers the SMs.
static int sapply_tensor_core(cpm_ctx* c, int nrep, cudaStream_t st) {
  CPM_CUDA(cudaMemsetAsync(c->qraw32, 0, sizeof(float) * (size_t)nrep * c->ne, st));
  const int mtiles = (c->ne + TC_M - 1) / TC_M;
  const int nchunks = (c->ld32 + TC_KC - 1) / TC_KC;
  const int splits = std::max(1, std::min(nchunks, (2 * 152 + mtiles - 1) / mtiles));
  const int cps = (nchunks + splits - 1) / splits;
  const dim3 grid(mtiles, (nchunks + cps - 1) / cps);
  for (int r0 = 0; r0 < nrep; r0 += 256) {
    const int left = nrep - r0;
    if (left <= 16) CPM_TRY(launch_tc<16>(c, r0, nrep, grid, cps, st));
    else if (left <= 32) CPM_TRY(launch_tc<32>(c, r0, nrep, grid, cps, st));
    else if (left <= 64) CPM_TRY(launch_tc<64>(c, r0, nrep, grid, cps, st));
    else if (left <= 128) CPM_TRY(launch_tc<128>(c, r0, nrep, grid, cps, st));
    else CPM_TRY(launch_tc<256>(c, r0, nrep, grid, cps, st));
  }
  return CPM_OK;
}

// Streaming S-apply of one block of rows (one replica) followed by its finish kernel.
static int sapply_stream(cpm_ctx* c, const float* S, int rows, int ld, const float* xh, const float* xl,
                         double* qpart, const double* b, const double* dpsi, const double* Sv, const double* W,
                         const double* c1, double* qout, cudaStream_t st) {
  const size_t smem = sizeof(float) * 2 * (size_t)ld;
  if (c->sapply_variant == CPM_SAPPLY_STREAM16)
    CPM_CUDA(launch_pdl(k_sapply_stream<16>, c->n_sm, SS_THREADS, smem, st, S, ld, rows, xh, xl, qpart));
  else
    CPM_CUDA(launch_pdl(k_sapply_stream<8>, c->n_sm, SS_THREADS, smem, st, S, ld, rows, xh, xl, qpart));
  STEP_LAUNCH();
  CPM_CUDA(launch_pdl(k_sapply_finish, (rows + FIN_THREADS - 1) / FIN_THREADS, FIN_THREADS, 0, st, rows, qpart, b, dpsi, Sv, W, c1, qout, c->scal));
  STEP_LAUNCH();
  return CPM_OK;
}

// One real-space pair launch with the context's kernel variant (cpm_pair_variant).
// elec_targets: the electrode-target kernels (real-space b, electrode forces) rather than the
// electrolyte-target ones; each kind follows its bit of the variant mask.
template <typename T, bool FORCE, bool LJ>
static int launch_pair(cpm_ctx* c, bool elec_targets, const CellPairTgt& tg, const PairSrc& a_in, const PairSrc& e_in,
                       const CellGeom& g, int nrep, int max_targets, const PairLj& lj, cudaStream_t s) {
  PairSrc a = a_in, e = e_in;
  a.beta_f = (float)a.beta;
  e.beta_f = (float)e.beta;
  using V4 = typename Vec4<T>::type;
  using V2 = typename Vec2<T>::type;
  const int bit = elec_targets ? CPM_PAIR_WARP_ELEC : CPM_PAIR_WARP_ELYT;
  if (c->pair_variant & bit) {
    const size_t smem = PW_WARPS * pw_warp_bytes<T>(g.nsten);
    const int blocks = std::max(1, std::min((max_targets + PW_WARPS - 1) / PW_WARPS, c->n_sm * 8));
    CPM_CUDA(launch_pdl(k_pair_warp<T, FORCE, LJ>, dim3(blocks, nrep), PW_THREADS, smem, s, tg, a, e, g, c->p.alpha,
                        c->scal, lj));
  } else {
    const size_t smem = (sizeof(V4) + (LJ ? sizeof(V2) : 0)) * kPairSrcCap;
    CPM_CUDA(launch_pdl(k_pair_cell<T, FORCE, LJ>, dim3(pair_blocks(g), nrep), PC_THREADS, smem, s, tg, a, e, g,
                        c->p.alpha, kPairSrcCap, c->scal, lj));
  }
  ++c->launches;
  CPM_LAUNCH();
  return CPM_OK;
}

// The third-law cell kernel for electrolyte targets (float32): one block per target-cell group.
static int launch_pair_n3(cpm_ctx* c, const CellPairTgt& tg, const PairSrc& a_in, const PairSrc& e_in,
                          const CellGeom& g_in, int nrep, cudaStream_t s) {
  PairSrc a = a_in, e = e_in;
  a.beta_f = (float)a.beta;
  e.beta_f = (float)e.beta;
  const CellGeom& g = g_in;
  const size_t smem = sizeof(float4) * kPairSrcCapN3;
  CPM_CUDA(launch_pdl(k_pair_cell<float, true, false, true>, dim3(pair_blocks(g), nrep), PC_THREADS, smem, s, tg,
                      a, e, g, c->p.alpha, kPairSrcCapN3, c->scal, PairLj{}));
  ++c->launches;
  CPM_LAUNCH();
  return CPM_OK;
}

template <typename T>
static int run(cpm_ctx* c, int nrep, const int* off, const double* xyzq, const double* dpsi, bool charges,
               double* q, double* b_out, double* psibar, double* f_elyt, double* f_elec, double* energy,
               cudaStream_t st) {
  using V4 = typename Vec4<T>::type;
  const int ne = c->ne, cap = c->p.max_elyt;
  const CellGeom g = cell_geom(c);
  const SpmeGeom sg = spme_geom(c);
  const double slab_coef = (c->p.geometry == CPM_SLAB) ? KE * 4.0 * PI / c->V : 0.0;
  const double ff_over_lz = (c->p.geometry == CPM_FF) ? 1.0 / c->Lz : 0.0;
  const V4* e_loc = c->mixed ? (const V4*)c->e_loc32 : (const V4*)c->e_loc64;
  V4* l_loc = c->mixed ? (V4*)c->l_loc32 : (V4*)c->l_loc64;
  V4* l_tmp = (V4*)c->l_tmp;
  T* qT = (T*)c->qT;
  const T* e_th = c->mixed ? (const T*)c->e_th32 : (const T*)c->e_th64;
  const T* e_dth = c->mixed ? (const T*)c->e_dth32 : (const T*)c->e_dth64;
  const T* splF = c->mixed ? (const T*)c->spl_F32 : (const T*)c->spl_F64;
  const dim3 gsite((cap + 255) / 256, nrep);
  const int sb = site_batch(c, cap, nrep);        // electrolyte sites per warp-batch of the mesh kernels

  const bool fork = c->prof_cap == 0;      // the profiler times phases one after another
  cudaStream_t sside = fork ? c->side : st;
  // brick charge assignment / interpolation (float32 mesh, sorted sites, TMA)
  const bool brick = c->mixed && c->brick_ok && c->mesh_variant == CPM_MESH_BRICK;
  // ---- prepare: cell list ----
  {
    PhaseTimer pt(c, st, CPM_PH_CELL_LIST);
    CPM_CUDA(cudaMemsetAsync(c->scal, 0, sizeof(double) * NSCAL * nrep, st));
    CPM_CUDA(cudaMemsetAsync(c->l_count, 0, sizeof(int) * (size_t)c->ncell * nrep, st));
    CPM_CUDA(launch_pdl(k_bin<T>, gsite, 256, 0, st, off, xyzq, cap, g, c->Lz, c->l_cell, c->l_count, l_tmp, c->ncell, c->scal,
                                    c->status));
    STEP_LAUNCH();
    // The sorted cell list serves only the real-space pair kernels, which run on the side stream:
    // fork here, so the counting sort overlaps the mesh work on the main stream (which reads k_bin's
    // per-site arrays).  Joined before the first main-stream use of the sorted arrays.
    if (fork) {
      CPM_CUDA(cudaEventRecord(c->ev_fork, st));
      CPM_CUDA(cudaStreamWaitEvent(c->side, c->ev_fork, 0));
    }
    CPM_CUDA(launch_pdl(k_scan, nrep, 1024, 0, sside, c->l_count, c->l_start, c->ncell));
    STEP_LAUNCH();
    CPM_CUDA(launch_pdl(k_scatter<T>, gsite, 256, 0, sside, off, cap, c->l_cell, l_tmp, c->l_count, c->ncell, c->l_sorted, l_loc));
    STEP_LAUNCH();
    if (fork) {
      CPM_CUDA(cudaEventRecord(c->ev_sorted, c->side));
      CPM_CUDA(cudaEventRecord(c->ev_join, c->side));
    }
  }

  PairSrc src_elyt{l_loc, (long long)cap, c->l_start, (long long)c->ncell + 1, c->l_sorted, nullptr, 0, 0.0, -1};
  PairSrc src_elec{e_loc, 0, c->e_start, 0, c->e_sorted, nullptr, ne, 0.0, -1};
  PairSrc none{nullptr, 0, nullptr, 0, nullptr, nullptr, 0, 0.0, -1};
  const size_t mesh_bytes = sizeof(T) * (size_t)c->Mr_s * nrep;

  // closed-form energy when the charges are solved in this call (cpm_step): U_elyt - q^T b / 2 + dpsi q^T v / 2
  const bool closed_form = charges && energy != nullptr;
  // electrolyte real-space field at the electrode sites from the b pass (electrode forces of cpm_step)
  const bool elec_field = charges && f_elec != nullptr && c->e_field != nullptr;

  if (charges) {
    double* b = c->b_tmp;                 // aligned internal copy, row stride ldb
    const int ldb = c->ldb;
    // real-space Gaussian-point part of b at the electrode sites
    // (on the side stream, concurrent with the mesh chain below; joined before the gather).  When
    // electrode forces follow in this call, the same pairs also give the electrolyte's real-space
    // field at the electrode sites: the electrode force is its charge times that field, so the
    // force pass needs no second sweep over these pairs.
    CellPairTgt tg{e_loc, 0, c->e_start, 0, c->e_sorted, ne, nullptr, nullptr, c->phi_real,
                   elec_field ? c->e_field : nullptr};
    PairSrc s = src_elyt;
    s.beta = c->p.eta;
    {
      PhaseTimer pt(c, st, CPM_PH_B_REAL);
      if (elec_field)
        CPM_TRY((launch_pair<T, true, false>(c, true, tg, s, none, g, nrep, ne, PairLj{}, sside)));
      else
        CPM_TRY((launch_pair<T, false, false>(c, true, tg, s, none, g, nrep, ne, PairLj{}, sside)));
    }
    if (fork) CPM_CUDA(cudaEventRecord(c->ev_join, c->side));
    // SPME part
    {
      PhaseTimer pt(c, st, CPM_PH_B_SPREAD);
      if (brick) {
        if (fork) CPM_CUDA(cudaStreamWaitEvent(st, c->ev_sorted, 0));
        CPM_TRY(cpm_internal_spread_brick(c, nrep, l_loc, nullptr, st));
      } else {
        CPM_CUDA(cudaMemsetAsync(c->mesh_r, 0, mesh_bytes, st));
        CPM_CUDA(launch_pdl(k_spread_elyt<T>, dim3(grid_for((cap + sb - 1) / sb), nrep), 256, 0, st, sb, off, cap, sg,
                            l_tmp, c->l_cell, c->spl_I, splF, (T*)c->mesh_r));
        STEP_LAUNCH();
      }
    }
    {
      PhaseTimer pt(c, st, CPM_PH_B_FFT);
      CPM_TRY(convolve<T>(c, nrep, closed_form ? S_E_RECIP_L : -1, st));
    }
    if (fork) CPM_CUDA(cudaStreamWaitEvent(st, c->ev_join, 0));
    {
      PhaseTimer pt(c, st, CPM_PH_B_GATHER);
      const int grp = elec_group(c, ne, nrep);
      CPM_CUDA(launch_pdl(k_gather_b<T>, dim3(grid_for((ne + grp - 1) / grp), nrep), 256, 0, st, (const T*)c->mesh_phi, ne,
                          c->e_base, e_th, sg, c->phi_real, c->e_z, slab_coef, c->scal, b,
                          (c->mixed && !c->mirror) ? c->b32 : nullptr, c->ldx, ldb, grp));
      STEP_LAUNCH();
      if (b_out) {
        CPM_CUDA(cudaMemcpy2DAsync(b_out, sizeof(double) * ne, b, sizeof(double) * ldb, sizeof(double) * ne, nrep,
                                   cudaMemcpyDeviceToDevice, st));
      }
    }
    // q = S b + dpsi S v, then the projection
    // one S-apply over `rows` rows of S (leading dimension ld), inputs x (float32 hi / lo halves or
    // float64 y), outputs q_raw rows of stride qstride
    auto sapply = [&](const float* S32, const double* S64, int rows, int ld, const float* x32, int xstride,
                      int xlo, const double* y64, int ldy, const double* Sv, const double* W, const double* c1,
                      double* qout, int qstride) -> int {
      const int sblocks = std::min(grid_for(rows), 152 * 4);
      for (int r0 = 0; r0 < nrep; r0 += 4) {
        const int left = nrep - r0;
        if (c->mixed) {
          if (left == 1)
            CPM_CUDA(launch_pdl(k_sapply32<1>, sblocks, 256, 0, st, S32, ld, rows, x32, xstride, xlo, y64, ldy, r0, nrep, dpsi, Sv,
                                                   W, c1, qout, qstride, c->scal));
          else if (left == 2)
            CPM_CUDA(launch_pdl(k_sapply32<2>, sblocks, 256, 0, st, S32, ld, rows, x32, xstride, xlo, y64, ldy, r0, nrep, dpsi, Sv,
                                                   W, c1, qout, qstride, c->scal));
          else
            CPM_CUDA(launch_pdl(k_sapply32<4>, sblocks, 256, 0, st, S32, ld, rows, x32, xstride, xlo, y64, ldy, r0, nrep, dpsi, Sv,
                                                   W, c1, qout, qstride, c->scal));
        } else {
          if (left == 1)
            CPM_CUDA(launch_pdl(k_sapply64<1>, sblocks, 256, 0, st, S64, ld, rows, y64, ldy, r0, nrep, dpsi, Sv, W, c1, qout,
                                                   qstride, c->scal));
          else if (left == 2)
            CPM_CUDA(launch_pdl(k_sapply64<2>, sblocks, 256, 0, st, S64, ld, rows, y64, ldy, r0, nrep, dpsi, Sv, W, c1, qout,
                                                   qstride, c->scal));
          else
            CPM_CUDA(launch_pdl(k_sapply64<4>, sblocks, 256, 0, st, S64, ld, rows, y64, ldy, r0, nrep, dpsi, Sv, W, c1, qout,
                                                   qstride, c->scal));
        }
        STEP_LAUNCH();
      }
      return CPM_OK;
    };
    // streaming variant: mixed precision, one replica, right-hand side fits shared memory
    const bool stream_ok = c->mixed && nrep == 1 && c->qpart &&
                           (c->sapply_variant == CPM_SAPPLY_STREAM || c->sapply_variant == CPM_SAPPLY_STREAM16);
    const bool sym_ok = c->mixed && nrep == 1 && c->sym_ok &&
                        (c->sapply_variant == CPM_SAPPLY_SYM || c->sapply_variant == CPM_SAPPLY_SYM_TMA);
    // the packed S-apply forms the projection sums itself (no finish pass) when its CTAs have few tiles
    const bool sym_fuse = sym_ok && cpm_internal_sym_fuse(c);
    {
      PhaseTimer pt(c, st, CPM_PH_S_APPLY);
      if (c->mirror) {
        const int nh = c->nh, ldh = c->ldh;
        CPM_CUDA(launch_pdl(k_mirror_fold, dim3((nh + 255) / 256, nrep), 256, 0, st, b, ldb, nh, ldh, c->m_i0, c->m_j, c->ypm,
                                                                    c->mixed ? c->b32 : nullptr));
        STEP_LAUNCH();
        for (int blk = 0; blk < 2; ++blk) {
          const size_t so = (size_t)blk * nh * ldh;
          if (sym_ok) {
            CPM_TRY(cpm_internal_sapply_sym(c, blk, c->b32 + (size_t)blk * ldh,
                                            c->b32 + 2 * (size_t)ldh + (size_t)blk * ldh, c->ypm + (size_t)blk * ldh,
                                            dpsi, c->Sv + (size_t)blk * nh, c->W + (size_t)blk * 2 * nh,
                                            c->e_c1m + (size_t)blk * nh, c->qpm + (size_t)blk * nh, st, sym_fuse));
            continue;
          }
          if (stream_ok) {
            CPM_TRY(sapply_stream(c, c->S32 + so, nh, ldh, c->b32 + (size_t)blk * ldh,
                                  c->b32 + 2 * (size_t)ldh + (size_t)blk * ldh, c->qpart + (size_t)blk * nh,
                                  c->ypm + (size_t)blk * ldh, dpsi, c->Sv + (size_t)blk * nh,
                                  c->W + (size_t)blk * 2 * nh, c->e_c1m + (size_t)blk * nh, c->qpm + (size_t)blk * nh,
                                  st));
            continue;
          }
          CPM_TRY(sapply(c->mixed ? c->S32 + so : nullptr, c->mixed ? nullptr : c->S64 + so, nh, ldh,
                         c->b32 + (size_t)blk * ldh, 4 * ldh, 2 * ldh, c->ypm + (size_t)blk * ldh, 2 * ldh,
                         c->Sv + (size_t)blk * nh, c->W + (size_t)blk * 2 * nh, c->e_c1m + (size_t)blk * nh,
                         c->qpm + (size_t)blk * nh, 2 * nh));
        }
      } else if (sym_ok) {
        CPM_TRY(cpm_internal_sapply_sym(c, 0, c->b32, c->b32 + c->ldx, b, dpsi, c->Sv, c->W, c->e_c1, q, st, sym_fuse));
      } else if (stream_ok) {
        CPM_TRY(sapply_stream(c, c->S32, ne, c->ld32, c->b32, c->b32 + c->ldx, c->qpart, b, dpsi, c->Sv, c->W, c->e_c1,
                              q, st));
      } else if (c->mixed && nrep >= TC_MIN_REPLICAS) {
        CPM_TRY(sapply_tensor_core(c, nrep, st));
        CPM_CUDA(launch_pdl(k_qraw_epilogue, dim3((ne + 255) / 256, nrep), 256, 0, st, c->qraw32, ne, b, ldb, dpsi, c->Sv, c->W,
                                                                      c->e_c1, q, c->scal));
        STEP_LAUNCH();
      } else {
        CPM_TRY(sapply(c->S32, c->S64, ne, c->ld64, c->b32, 2 * c->ldx, c->ldx, b, ldb, c->Sv, c->W, c->e_c1, q,
                       ne));
      }
    }
    PhaseTimer ptp(c, st, CPM_PH_PROJECT);
    // when the force pass follows, the projection also leaves the charges in its working precision
    // and their sums (the work of k_charge_prep)
    const bool forces_follow = f_elyt || f_elec || energy;
    const ChargePrep<T> cprep{forces_follow ? qT : nullptr, c->e_z, c->e_v, c->e_plus};
    // after the packed S-apply with its own sums the projection reads its row accumulator
    // (q_raw - dpsi S v)
    const QRawPart qp{sym_fuse ? c->qpart : nullptr, c->Sv, c->sym_sv[0], c->sym_sv[1]};
    if (c->mirror) {
      CPM_CUDA(launch_pdl(k_project_mirror<T>, dim3((c->nh + FIN_THREADS - 1) / FIN_THREADS, nrep), FIN_THREADS, 0, st, c->qpm, c->nh, c->m_i0, c->m_j, c->W, b,
                                                                        ldb, ne, c->scal, dpsi, c->Mh[0], c->Mh[1],
                                                                        c->WTv[0], c->WTv[1], q, psibar, cprep, qp));
    } else {
      CPM_CUDA(launch_pdl(k_project<T>, dim3((ne + FIN_THREADS - 1) / FIN_THREADS, nrep), FIN_THREADS, 0, st, q, ne, nrep, c->ncons, c->W, b, ldb, c->scal, dpsi,
                                                              c->Mh[0], c->Mh[1], c->Mh[2], c->Mh[3], c->WTv[0],
                                                              c->WTv[1], psibar, cprep, qp));
    }
    STEP_LAUNCH();
  }

  if (f_elyt || f_elec || energy) {
    cudaStream_t sp = sside;
    // electrolyte forces by the third-law cell kernel (CPM_PAIR_N3_ELYT; mixed precision, not in an
    // MD loop with Lennard-Jones, site charge assignment): into the float32 sorted-order buffer
    const bool n3 = f_elyt != nullptr && c->lj == nullptr && c->mixed && (c->pair_variant & CPM_PAIR_N3_ELYT) &&
                    !(c->pair_variant & CPM_PAIR_WARP_ELYT) && !brick && c->f_sorted32 != nullptr;
    if (!charges) {                      // charges given by the caller (cpm_forces, cpm_energy)
      PhaseTimer pt(c, st, CPM_PH_F_SPREAD);
      CPM_CUDA(launch_pdl(k_charge_prep<T>, dim3((ne + 255) / 256, nrep), 256, 0, st, q, ne, c->e_z, c->e_v, c->e_plus, qT, c->scal));
      STEP_LAUNCH();
    }
    // Electrode-electrode forces of the frozen electrode from the pair list precomputed at build
    // (mixed precision, forces without the full-sum energy).  In cpm_step they are added to the
    // electrolyte field of the b pass, on the side stream ahead of the electrolyte pair forces,
    // and the electrode gather forms q_i times the total field; otherwise they are added to the
    // forces after the gather.
    const bool ee_list = (c->ee_g != nullptr || c->ee_idx != nullptr) && f_elec && !(energy && !closed_form) &&
                         sizeof(T) == sizeof(float);
    const bool ee_field = ee_list && elec_field;
    auto launch_ee = [&](cudaStream_t s_ee, double* dst, int mulq) -> int {
      if (c->ee_idx) {
        // 8 lanes per row when the rows fill the resident warps, else 32 (chosen at build, which
        // orders the entries for it); row groups of 4 or 1 rows per warp pass
        const bool wide = c->ee_lpr == 32;
        const int rpp = wide ? 1 : 4;
        const int grp = std::max(rpp, (elec_group(c, ne, nrep) + rpp - 1) / rpp * rpp);
        const int blocks = std::max(1, std::min((ne + 8 * grp - 1) / (8 * grp), c->n_sm * 8));
        const size_t smem = sizeof(float4) * (size_t)c->ee_ntab;
        if (wide)
          CPM_CUDA(launch_pdl(k_ee_forces_tab<32>, dim3(blocks, nrep), 256, smem, s_ee, (const int*)c->ee_ptr,
                              (const uint4*)c->ee_idx, (const float4*)c->ee_tab, c->ee_ntab, ne, (const float*)qT,
                              dst, grp, mulq));
        else
          CPM_CUDA(launch_pdl(k_ee_forces_tab<8>, dim3(blocks, nrep), 256, smem, s_ee, (const int*)c->ee_ptr,
                              (const uint4*)c->ee_idx, (const float4*)c->ee_tab, c->ee_ntab, ne, (const float*)qT,
                              dst, grp, mulq));
      } else {
        const int grp = elec_group(c, ne, nrep);
        const int blocks = std::max(1, std::min((ne + 8 * grp - 1) / (8 * grp), c->n_sm * 8));
        CPM_CUDA(launch_pdl(k_ee_forces, dim3(blocks, nrep), 256, 0, s_ee, (const int*)c->ee_ptr,
                            (const float4*)c->ee_g, ne, (const float*)qT, dst, grp, mulq));
      }
      STEP_LAUNCH();
      return CPM_OK;
    };
    // real space, electrolyte targets: point-point (elyt) + Gaussian-point (electrodes), into f_pair;
    // on the side stream, concurrent with the mesh chain, joined before the force gather
    if (fork) {
      CPM_CUDA(cudaEventRecord(c->ev_fork, st));
      CPM_CUDA(cudaStreamWaitEvent(c->side, c->ev_fork, 0));
    }
    if (ee_field) {
      PhaseTimer pt(c, st, CPM_PH_F_PAIR_ELEC);
      CPM_TRY(launch_ee(sp, c->e_field, 0));
      if (fork) CPM_CUDA(cudaEventRecord(c->ev_ee, c->side));
    }
    {
      PhaseTimer pt(c, st, CPM_PH_F_PAIR_ELYT);
      if (f_elyt && !n3) CPM_CUDA(cudaMemsetAsync(c->f_pair, 0, sizeof(double) * 3 * (size_t)cap * nrep, sp));
      if (n3) CPM_CUDA(cudaMemsetAsync(c->f_sorted32, 0, sizeof(float) * 3 * (size_t)cap * nrep, sp));
      CellPairTgt tg{l_loc, (long long)cap, c->l_start, (long long)c->ncell + 1, c->l_sorted, cap, nullptr,
                     (f_elyt && !n3) ? c->f_pair : nullptr, nullptr, nullptr, n3 ? c->f_sorted32 : nullptr};
      PairSrc a = src_elyt;
      a.slot = S_E_LL;
      PairSrc e = src_elec;
      e.qT = qT;
      e.beta = c->p.eta;
      e.slot = closed_form ? -1 : S_E_LE;         // the closed-form energy does not use it
      if (f_elyt && c->lj) {
        // Lennard-Jones of a running MD loop, fused: the same staged sources and pair list
        PairLj lj;
        lj.type = c->lj->type;
        lj.off = off;
        lj.elec_type = c->lj->elec_type;
        lj.cut = c->lj->cut;
        for (int k = 0; k < kLjMaxTypes; ++k) {
          lj.sig_half[k] = c->lj->sig_half[k];
          lj.sqrt_eps[k] = c->lj->sqrt_eps[k];
        }
        CPM_TRY((launch_pair<T, true, true>(c, false, tg, a, e, g, nrep, cap, lj, sp)));
      } else if (n3) {
        CPM_TRY(launch_pair_n3(c, tg, a, e, g, nrep, sp));
      } else if (f_elyt) {
        CPM_TRY((launch_pair<T, true, false>(c, false, tg, a, e, g, nrep, cap, PairLj{}, sp)));
      } else {
        CPM_TRY((launch_pair<T, false, false>(c, false, tg, a, e, g, nrep, cap, PairLj{}, sp)));
      }
    }
    if (fork) CPM_CUDA(cudaEventRecord(c->ev_join, c->side));
    // SPME of all charges
    {
      PhaseTimer pt(c, st, CPM_PH_F_SPREAD);
      if (brick) {
        if (fork) CPM_CUDA(cudaStreamWaitEvent(st, c->ev_sorted, 0));
        CPM_TRY(cpm_internal_spread_brick(c, nrep, l_loc, (const float*)qT, st));
      } else {
        CPM_CUDA(cudaMemsetAsync(c->mesh_r, 0, mesh_bytes, st));
        const int nb_l = grid_for((cap + sb - 1) / sb), nb_e = grid_for(ne);
        // electrolyte sites in cell-sorted order: neighbouring sites' atomics hit the same lines
        // (the sorted list reached the main stream at the b pass's join; in a call without
        // charges the join comes below, so input order is used there)
        const bool sorted_ok = charges || !fork;
        CPM_CUDA(launch_pdl(k_spread_all<T>, dim3(nb_l + nb_e, nrep), 256, 0, st, nb_l, sb, off, cap, sg,
                            sorted_ok ? (const V4*)l_loc : (const V4*)l_tmp, c->l_cell, c->spl_I, splF, qT, ne,
                            c->e_base, e_th, (T*)c->mesh_r, sorted_ok ? (const int*)c->l_sorted : nullptr));
        STEP_LAUNCH();
      }
    }
    {
      PhaseTimer pt(c, st, CPM_PH_F_FFT);
      CPM_TRY(convolve<T>(c, nrep, (energy && !closed_form) ? S_E_RECIP : -1, st));
    }
    PhaseTimer ptg(c, st, CPM_PH_F_GATHER);
    // electrode sites first: they wait only for the pair-list field (when it is used), not for
    // the electrolyte pair forces
    if (f_elec) {
      if (fork && ee_field) CPM_CUDA(cudaStreamWaitEvent(st, c->ev_ee, 0));
      const int grp = elec_group(c, ne, nrep);
      CPM_CUDA(launch_pdl(k_gather_f_elec<T>, dim3(grid_for((ne + grp - 1) / grp), nrep), 256, 0, st, (const T*)c->mesh_phi, qT,
                          ne, c->e_base, e_th, e_dth, sg, dpsi, ff_over_lz, slab_coef, c->scal,
                          elec_field ? (const double*)c->e_field : nullptr, f_elec, grp));
      STEP_LAUNCH();
    }
    // electrolyte sites in cell-sorted order.  With the side stream, the mesh part is gathered
    // while the pair kernels still run (it needs only the sorted list: joined in the b pass, or
    // waited for here), and the real-space forces are added after the join; without it (the
    // profiler's serial phases), in one pass
    if (f_elyt && !brick) {
      if (fork && !charges) CPM_CUDA(cudaStreamWaitEvent(st, c->ev_sorted, 0));
      CPM_CUDA(launch_pdl(k_gather_f_elyt<T>, dim3(grid_for((cap + sb - 1) / sb), nrep), 256, 0, st, sb,
                          (const T*)c->mesh_phi, off, cap, sg, (const V4*)l_loc, c->l_cell, c->spl_I, splF, dpsi,
                          ff_over_lz, slab_coef, c->scal, fork ? nullptr : (const double*)c->f_pair,
                          (!fork && n3) ? (const float*)c->f_sorted32 : nullptr, f_elyt, (const int*)c->l_sorted));
      STEP_LAUNCH();
    }
    if (fork) CPM_CUDA(cudaStreamWaitEvent(st, c->ev_join, 0));
    if (f_elyt && brick) {
      CPM_TRY(cpm_internal_gather_f_brick(c, nrep, off, l_loc, dpsi, ff_over_lz, slab_coef, f_elyt, st));
    } else if (f_elyt && fork) {
      CPM_CUDA(launch_pdl(k_add_pair_forces, dim3((cap + 255) / 256, nrep), 256, 0, st, off, cap,
                          (const int*)c->l_sorted, n3 ? nullptr : (const double*)c->f_pair,
                          n3 ? (const float*)c->f_sorted32 : nullptr, f_elyt));
      STEP_LAUNCH();
    }
    ptg.stop();
    // real space, electrode targets: Gaussian-point (forces only, unless the b pass gave the field)
    // + Gaussian-Gaussian (forces, and the energy of the full sum) unless the pair list gives them
    if (f_elec || (energy && !closed_form)) {
      CellPairTgt tg{e_loc, 0, c->e_start, 0, c->e_sorted, ne, qT, f_elec, nullptr, nullptr};
      PairSrc a = (f_elec && !elec_field) ? src_elyt : none;
      a.beta = c->p.eta;
      PairSrc e = src_elec;
      e.qT = qT;
      e.beta = c->p.eta / std::sqrt(2.0);
      e.slot = (energy && !closed_form) ? S_E_EE : -1;
      if (ee_list) e = none;
      const bool ee_late = ee_list && !ee_field;
      if (a.loc != nullptr || e.loc != nullptr || ee_late) {
        PhaseTimer pt(c, st, CPM_PH_F_PAIR_ELEC);
        if (a.loc == nullptr && e.loc == nullptr) {
          // the pair list alone
        } else if (f_elec) {
          CPM_TRY((launch_pair<T, true, false>(c, true, tg, a, e, g, nrep, ne, PairLj{}, st)));
        } else {
          CPM_TRY((launch_pair<T, false, false>(c, true, tg, a, e, g, nrep, ne, PairLj{}, st)));
        }
        if (ee_late) CPM_TRY(launch_ee(st, f_elec, 1));
      }
    }
    if (energy) {
      PhaseTimer pt(c, st, CPM_PH_ENERGY);
      const double slab_e = (c->p.geometry == CPM_SLAB) ? KE * 2.0 * PI / c->V : 0.0;
      CPM_CUDA(launch_pdl(k_energy_final, (nrep + 127) / 128, 128, 0, st, nrep, c->scal, dpsi, c->p.alpha, c->p.eta, slab_e,
                                                         ff_over_lz, closed_form ? 1 : 0, energy));
      STEP_LAUNCH();
    }
  }
  // every side-stream branch ends joined into the caller's stream (required to end a capture)
  if (fork) {
    CPM_CUDA(cudaEventRecord(c->ev_join, c->side));
    CPM_CUDA(cudaStreamWaitEvent(st, c->ev_join, 0));
  }
  return CPM_OK;
}

static int dispatch(cpm_ctx* c, int nrep, const int* off, const double* xyzq, const double* dpsi, bool charges,
                    double* q, double* b, double* psibar, double* f_elyt, double* f_elec, double* energy,
                    void* stream) {
  if (!c || !off || !xyzq || !dpsi || !q) {
    set_error("null context or required pointer");
    return CPM_ERR_ARG;
  }
  if (nrep < 1 || nrep > c->p.max_replicas) {
    set_error("n_rep %d outside [1, %d]", nrep, c->p.max_replicas);
    return CPM_ERR_CAPACITY;
  }
  if (reinterpret_cast<uintptr_t>(xyzq) % 32 != 0) {
    set_error("elyt_xyzq_dev must be 32-byte aligned");
    return CPM_ERR_ARG;
  }
  cudaStream_t st = (cudaStream_t)stream;
  return c->mixed ? run<float>(c, nrep, off, xyzq, dpsi, charges, q, b, psibar, f_elyt, f_elec, energy, st)
                  : run<double>(c, nrep, off, xyzq, dpsi, charges, q, b, psibar, f_elyt, f_elec, energy, st);
}

}  // namespace cpm

// The float64 cell-block pair kernel stages 64 KiB of sources: raise its dynamic shared memory limit.
static int pair_cell_attributes() {
  const int d64 = (int)(sizeof(double4_32a) * cpm::kPairSrcCap), d32 = (int)(sizeof(float4) * cpm::kPairSrcCap);
  CPM_CUDA(cudaFuncSetAttribute(cpm::k_pair_cell<double, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, d64));
  CPM_CUDA(cudaFuncSetAttribute(cpm::k_pair_cell<double, false>, cudaFuncAttributeMaxDynamicSharedMemorySize, d64));
  CPM_CUDA(cudaFuncSetAttribute(cpm::k_pair_cell<float, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, d32));
  CPM_CUDA(cudaFuncSetAttribute(cpm::k_pair_cell<float, false>, cudaFuncAttributeMaxDynamicSharedMemorySize, d32));
  CPM_CUDA(cudaFuncSetAttribute(cpm::k_pair_cell<float, true, false, true>,
                                cudaFuncAttributeMaxDynamicSharedMemorySize, d32));
  const int l64 = (int)((sizeof(double4_32a) + sizeof(double2)) * cpm::kPairSrcCap);
  const int l32 = (int)((sizeof(float4) + sizeof(float2)) * cpm::kPairSrcCap);
  CPM_CUDA(cudaFuncSetAttribute(cpm::k_pair_cell<double, true, true>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                l64));
  CPM_CUDA(cudaFuncSetAttribute(cpm::k_pair_cell<float, true, true>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                l32));
  // warp-per-target variant: per-warp stencil tables for the largest stencil
  const int w64 = (int)(cpm::PW_WARPS * cpm::pw_warp_bytes<double>(cpm::kMaxStencil));
  const int w32 = (int)(cpm::PW_WARPS * cpm::pw_warp_bytes<float>(cpm::kMaxStencil));
  CPM_CUDA(cudaFuncSetAttribute(cpm::k_pair_warp<double, false, false>, cudaFuncAttributeMaxDynamicSharedMemorySize, w64));
  CPM_CUDA(cudaFuncSetAttribute(cpm::k_pair_warp<double, true, false>, cudaFuncAttributeMaxDynamicSharedMemorySize, w64));
  CPM_CUDA(cudaFuncSetAttribute(cpm::k_pair_warp<double, true, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, w64));
  CPM_CUDA(cudaFuncSetAttribute(cpm::k_pair_warp<float, false, false>, cudaFuncAttributeMaxDynamicSharedMemorySize, w32));
  CPM_CUDA(cudaFuncSetAttribute(cpm::k_pair_warp<float, true, false>, cudaFuncAttributeMaxDynamicSharedMemorySize, w32));
  CPM_CUDA(cudaFuncSetAttribute(cpm::k_pair_warp<float, true, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, w32));
  // compressed electrode pair list: the table of distinct G vectors
  const int et = (int)(sizeof(float4) * cpm::kEeTabMax);
  CPM_CUDA(cudaFuncSetAttribute(cpm::k_ee_forces_tab<8>, cudaFuncAttributeMaxDynamicSharedMemorySize, et));
  CPM_CUDA(cudaFuncSetAttribute(cpm::k_ee_forces_tab<32>, cudaFuncAttributeMaxDynamicSharedMemorySize, et));
  return CPM_OK;
}

static int tc_attributes() {
  CPM_CUDA(cudaFuncSetAttribute(cpm::k_sapply_tc<16>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                (int)cpm::tc_smem_bytes<16>()));
  CPM_CUDA(cudaFuncSetAttribute(cpm::k_sapply_tc<32>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                (int)cpm::tc_smem_bytes<32>()));
  CPM_CUDA(cudaFuncSetAttribute(cpm::k_sapply_tc<64>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                (int)cpm::tc_smem_bytes<64>()));
  CPM_CUDA(cudaFuncSetAttribute(cpm::k_sapply_tc<128>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                (int)cpm::tc_smem_bytes<128>()));
  CPM_CUDA(cudaFuncSetAttribute(cpm::k_sapply_tc<256>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                (int)cpm::tc_smem_bytes<256>()));
  return CPM_OK;
}

static bool stream_available(const cpm_ctx* c) {
  return c->mixed && sizeof(float) * 2 * (size_t)c->ld32 <= (size_t)cpm::SS_SMEM_MAX;
}

cpm::SpmeGeom cpm_internal_spme_geom(const cpm_ctx* c) { return cpm::spme_geom(c); }

// A z group of gz cells per pair-kernel block is possible while its stencil fits the kernel's tables.
static bool pair_group_ok(const cpm_ctx* c, int gz) {
  return gz >= 1 && gz <= 8 && (2 * c->sten[0] + 1) * (2 * c->sten[1] + 1) * (gz + 2 * c->sten[2]) <= cpm::kMaxStencil;
}

int cpm_internal_alloc_step_buffers(cpm_ctx* c) {
  CPM_TRY(pair_cell_attributes());
  CPM_TRY(tc_attributes());
  CPM_CUDA(cudaDeviceGetAttribute(&c->n_sm, cudaDevAttrMultiProcessorCount, c->dev));
  // one cell per pair-kernel block unless the autotuner finds a z group faster: the per-source
  // distance checks, not the staging the groups share, dominate the kernel (measured on GB300)
  c->pair_gz = 1;
  CPM_TRY(cpm_internal_fft_setup(c));
  CPM_TRY(cpm_internal_brick_setup(c));
  if (stream_available(c)) {
    CPM_CUDA(cudaFuncSetAttribute(cpm::k_sapply_stream<8>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                  cpm::SS_SMEM_MAX));
    CPM_CUDA(cudaFuncSetAttribute(cpm::k_sapply_stream<16>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                  cpm::SS_SMEM_MAX));
    const long long rows = c->mirror ? 2LL * c->nh : (long long)c->ne;
    CPM_CUDA(cudaMalloc(&c->qpart, sizeof(double) * rows));
    CPM_CUDA(cudaMemset(c->qpart, 0, sizeof(double) * rows));
    // default before any tuning: stream matrices well above the L2 capacity
    c->sapply_variant = (rows * c->ld32 * 4LL >= (64LL << 20)) ? CPM_SAPPLY_STREAM : CPM_SAPPLY_ROWS;
  }
  CPM_TRY(cpm_internal_sym_setup(c));          // after qpart: the packed S-apply adds into it
  const size_t R = c->p.max_replicas, cap = c->p.max_elyt, ne = c->ne;
  const size_t tsz = c->mixed ? sizeof(float) : sizeof(double);
  const size_t v4 = c->mixed ? sizeof(float4) : sizeof(double4_32a);
  CPM_CUDA(cudaMalloc(&c->mesh_r, tsz * c->Mr_s * R));
  CPM_CUDA(cudaMalloc(&c->mesh_phi, tsz * c->Mr_s * R));
  CPM_CUDA(cudaMalloc(&c->mesh_c, 2 * tsz * c->Mc_s * R));
  CPM_CUDA(cudaMalloc(&c->l_cell, sizeof(int) * R * cap));
  CPM_CUDA(cudaMalloc(&c->l_count, sizeof(int) * R * c->ncell));
  CPM_CUDA(cudaMalloc(&c->l_start, sizeof(int) * R * (c->ncell + 1)));
  CPM_CUDA(cudaMalloc(&c->l_sorted, sizeof(int) * R * cap));
  if (c->mixed)
    CPM_CUDA(cudaMalloc(&c->l_loc32, v4 * R * cap));
  else
    CPM_CUDA(cudaMalloc(&c->l_loc64, v4 * R * cap));
  CPM_CUDA(cudaMalloc(&c->l_tmp, v4 * R * cap));
  CPM_CUDA(cudaMalloc(&c->qT, tsz * R * ne));
  CPM_CUDA(cudaMalloc(&c->phi_real, sizeof(double) * R * ne));
  CPM_CUDA(cudaMalloc(&c->e_field, sizeof(double) * 3 * R * ne));
  CPM_CUDA(cudaMalloc(&c->b_tmp, sizeof(double) * R * c->ldb));
  CPM_CUDA(cudaMemset(c->b_tmp, 0, sizeof(double) * R * c->ldb));
  CPM_CUDA(cudaMalloc(&c->b32, sizeof(float) * R * 2 * c->ldx));
  CPM_CUDA(cudaMemset(c->b32, 0, sizeof(float) * R * 2 * c->ldx));
  if (c->mirror) {
    CPM_CUDA(cudaMalloc(&c->ypm, sizeof(double) * R * 2 * c->ldh));
    CPM_CUDA(cudaMemset(c->ypm, 0, sizeof(double) * R * 2 * c->ldh));
    CPM_CUDA(cudaMalloc(&c->qpm, sizeof(double) * R * 2 * c->nh));
  }
  CPM_CUDA(cudaMalloc(&c->f_pair, sizeof(double) * R * cap * 3));
  CPM_CUDA(cudaMalloc(&c->f_sorted32, sizeof(float) * R * cap * 3));
  CPM_CUDA(cudaStreamCreateWithFlags(&c->side, cudaStreamNonBlocking));
  CPM_CUDA(cudaEventCreateWithFlags(&c->ev_fork, cudaEventDisableTiming));
  CPM_CUDA(cudaEventCreateWithFlags(&c->ev_join, cudaEventDisableTiming));
  CPM_CUDA(cudaEventCreateWithFlags(&c->ev_sorted, cudaEventDisableTiming));
  CPM_CUDA(cudaEventCreateWithFlags(&c->ev_ee, cudaEventDisableTiming));
  CPM_CUDA(cudaMalloc(&c->scal, sizeof(double) * R * cpm::NSCAL));
  if (c->mixed && (int)R >= cpm::TC_MIN_REPLICAS) CPM_CUDA(cudaMalloc(&c->qraw32, sizeof(float) * R * ne));
  CPM_CUDA(cudaMalloc(&c->status, sizeof(int)));
  CPM_CUDA(cudaMemset(c->status, 0, sizeof(int)));
  CPM_TRY(cpm_internal_static_scratch_setup());
  return CPM_OK;
}

// ------------------------------------------------------------------------------------------
// C ABI
// ------------------------------------------------------------------------------------------
extern "C" int cpm_step_charges(cpm_ctx* ctx, int32_t n_rep, const int32_t* off, const double* xyzq,
                                const double* dpsi, double* q, double* b, double* psibar, void* stream) {
  return cpm::dispatch(ctx, n_rep, off, xyzq, dpsi, true, q, b, psibar, nullptr, nullptr, nullptr, stream);
}

extern "C" int cpm_forces(cpm_ctx* ctx, int32_t n_rep, const int32_t* off, const double* xyzq,
                          const double* dpsi, const double* q, double* f_elyt, double* f_elec, double* energy,
                          void* stream) {
  return cpm::dispatch(ctx, n_rep, off, xyzq, dpsi, false, const_cast<double*>(q), nullptr, nullptr, f_elyt,
                       f_elec, energy, stream);
}

extern "C" int cpm_energy(cpm_ctx* ctx, int32_t n_rep, const int32_t* off, const double* xyzq,
                          const double* dpsi, const double* q, double* energy, void* stream) {
  if (!energy) return CPM_ERR_ARG;
  return cpm::dispatch(ctx, n_rep, off, xyzq, dpsi, false, const_cast<double*>(q), nullptr, nullptr, nullptr,
                       nullptr, energy, stream);
}

extern "C" int cpm_step(cpm_ctx* ctx, int32_t n_rep, const int32_t* off, const double* xyzq, const double* dpsi,
                        double* q, double* psibar, double* f_elyt, double* f_elec, double* energy, void* stream) {
  return cpm::dispatch(ctx, n_rep, off, xyzq, dpsi, true, q, nullptr, psibar, f_elyt, f_elec, energy, stream);
}

extern "C" int cpm_set_sapply_variant(cpm_ctx* c, int32_t variant) {
  if (!c) return CPM_ERR_ARG;
  if (variant == CPM_SAPPLY_ROWS) {
    c->sapply_variant = variant;
    return CPM_OK;
  }
  if (((variant == CPM_SAPPLY_STREAM || variant == CPM_SAPPLY_STREAM16) && stream_available(c) && c->qpart) ||
      ((variant == CPM_SAPPLY_SYM || variant == CPM_SAPPLY_SYM_TMA) && c->sym_ok)) {
    c->sapply_variant = variant;
    return CPM_OK;
  }
  cpm::set_error("cpm_set_sapply_variant: variant %d is not available for this context", variant);
  return CPM_ERR_ARG;
}

extern "C" int cpm_set_pair_group(cpm_ctx* c, int32_t gz) {
  if (!c || !pair_group_ok(c, gz)) {
    cpm::set_error("cpm_set_pair_group: %d z cells per block is outside 1..8 or exceeds the stencil tables", gz);
    return CPM_ERR_ARG;
  }
  c->pair_gz = gz;
  return CPM_OK;
}

extern "C" int cpm_set_wait_test(cpm_ctx* c, int32_t on) {
  if (!c) {
    cpm::set_error("cpm_set_wait_test: null context");
    return CPM_ERR_ARG;
  }
  c->wait_test = on != 0;
  return CPM_OK;
}

extern "C" int cpm_get_pair_group(const cpm_ctx* c, int32_t* gz) {
  if (!c || !gz) return CPM_ERR_ARG;
  *gz = c->pair_gz;
  return CPM_OK;
}

extern "C" int cpm_set_pair_variant(cpm_ctx* c, int32_t variant) {
  if (!c || variant < CPM_PAIR_CELL || variant > (CPM_PAIR_N3_ELYT | CPM_PAIR_WARP_ELEC) ||
      ((variant & CPM_PAIR_N3_ELYT) && (variant & CPM_PAIR_WARP_ELYT))) {
    cpm::set_error("cpm_set_pair_variant: unknown variant %d", variant);
    return CPM_ERR_ARG;
  }
  c->pair_variant = variant;
  return CPM_OK;
}

extern "C" int cpm_get_pair_variant(const cpm_ctx* c, int32_t* variant) {
  if (!c || !variant) return CPM_ERR_ARG;
  *variant = c->pair_variant;
  return CPM_OK;
}

extern "C" int cpm_set_fft_variant(cpm_ctx* c, int32_t variant) {
  if (!c) return CPM_ERR_ARG;
  if (variant == CPM_FFT_LIBRARY || (variant == CPM_FFT_OWN && c->fft_own_ok)) {
    c->fft_variant = variant;
    return CPM_OK;
  }
  cpm::set_error("cpm_set_fft_variant: variant %d is not available for this context", variant);
  return CPM_ERR_ARG;
}

extern "C" int cpm_set_mesh_variant(cpm_ctx* c, int32_t variant) {
  if (!c) return CPM_ERR_ARG;
  if (variant == CPM_MESH_SITES || (variant == CPM_MESH_BRICK && c->brick_ok)) {
    c->mesh_variant = variant;
    return CPM_OK;
  }
  cpm::set_error("cpm_set_mesh_variant: variant %d is not available for this context", variant);
  return CPM_ERR_ARG;
}

extern "C" int cpm_autotune(cpm_ctx* c, const int32_t* off, const double* xyzq, const double* dpsi, double* q,
                            void* stream, int32_t* choice_host) {
  if (!c || !off || !xyzq || !dpsi || !q) return CPM_ERR_ARG;
  cudaStream_t st = (cudaStream_t)stream;
  const int keep_s = c->sapply_variant, keep_f = c->fft_variant, keep_m = c->mesh_variant, keep_g = c->pair_gz,
            keep_p = c->pair_variant;
  // every timed call starts from a cold L2 (a write of twice its capacity), as inside an MD step
  // whose other work evicts S
  int l2 = 0;
  CPM_CUDA(cudaDeviceGetAttribute(&l2, cudaDevAttrL2CacheSize, c->dev));
  const size_t flush_bytes = std::max<size_t>(2 * (size_t)l2, 64u << 20);
  void* flush = nullptr;
  CPM_CUDA(cudaMalloc(&flush, flush_bytes));
  cudaEvent_t e0, e1;
  CPM_CUDA(cudaEventCreate(&e0));
  CPM_CUDA(cudaEventCreate(&e1));
  int rc = CPM_OK;
  // scratch outputs of the timed steps (forces and energies are part of the step)
  double *f_scr = nullptr, *fe_scr = nullptr, *e_scr = nullptr;
  CPM_CUDA(cudaMalloc(&f_scr, sizeof(double) * 3 * (size_t)c->p.max_elyt + 64));
  CPM_CUDA(cudaMalloc(&fe_scr, sizeof(double) * 3 * (size_t)c->ne + 64));
  CPM_CUDA(cudaMalloc(&e_scr, sizeof(double) * cpm::NENERGY));
  // Each stage times its candidates, the current choice among them, as replays of CUDA graphs of
  // the whole step (charges, forces, energy) captured on a private stream, as the step runs in an
  // MD loop; without graphs (profiler on), direct calls.  The candidates' replays are interleaved
  // round by round, so that a drift of the clocks during the tuning biases none of them; each
  // candidate's median decides.
  cudaStream_t cs = nullptr;
  CPM_CUDA(cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking));
  const bool use_graph = c->prof_cap == 0;
  struct Cfg {
    int sv, fv, mv, gz, pv;
  };
  auto apply = [&](const Cfg& k) -> bool {
    if (cpm_set_sapply_variant(c, k.sv) != CPM_OK || cpm_set_fft_variant(c, k.fv) != CPM_OK ||
        cpm_set_mesh_variant(c, k.mv) != CPM_OK || !pair_group_ok(c, k.gz))
      return false;
    c->pair_gz = k.gz;
    c->pair_variant = k.pv;
    return true;
  };
  constexpr int ROUNDS = 15;
  auto choose = [&](const std::vector<Cfg>& cand, Cfg* best) {
    std::vector<Cfg> ok;
    std::vector<cudaGraph_t> gr;
    std::vector<cudaGraphExec_t> ge;
    for (const Cfg& k : cand) {
      if (rc != CPM_OK) break;
      if (!apply(k)) continue;
      rc = cpm_step(c, 1, off, xyzq, dpsi, q, nullptr, f_scr, fe_scr, e_scr, st);
      if (rc == CPM_OK && cudaStreamSynchronize(st) != cudaSuccess) rc = CPM_ERR_CUDA;
      if (rc != CPM_OK) break;
      cudaGraph_t g = nullptr;
      cudaGraphExec_t x = nullptr;
      if (use_graph) {
        if (cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal) != cudaSuccess) {
          rc = CPM_ERR_CUDA;
          break;
        }
        const int r2 = cpm_step(c, 1, off, xyzq, dpsi, q, nullptr, f_scr, fe_scr, e_scr, cs);
        const cudaError_t ec = cudaStreamEndCapture(cs, &g);
        if (r2 != CPM_OK) rc = r2;
        else if (ec != cudaSuccess || cudaGraphInstantiate(&x, g, 0) != cudaSuccess) rc = CPM_ERR_CUDA;
        if (rc != CPM_OK) {
          if (g) cudaGraphDestroy(g);
          break;
        }
      }
      ok.push_back(k);
      gr.push_back(g);
      ge.push_back(x);
    }
    std::vector<std::vector<float>> ms(ok.size());
    cudaStream_t ts = use_graph ? cs : st;
    for (int r = 0; r < ROUNDS + 1 && rc == CPM_OK; ++r) {      // round 0 warms up
      for (size_t i = 0; i < ok.size() && rc == CPM_OK; ++i) {
        if (!use_graph) apply(ok[i]);
        cudaMemsetAsync(flush, r, flush_bytes, ts);
        cudaEventRecord(e0, ts);
        if (use_graph) {
          if (cudaGraphLaunch(ge[i], ts) != cudaSuccess) rc = CPM_ERR_CUDA;
        } else {
          rc = cpm_step(c, 1, off, xyzq, dpsi, q, nullptr, f_scr, fe_scr, e_scr, ts);
        }
        cudaEventRecord(e1, ts);
        float t = 0.f;
        if (cudaEventSynchronize(e1) != cudaSuccess) rc = CPM_ERR_CUDA;
        else if (r > 0 && cudaEventElapsedTime(&t, e0, e1) == cudaSuccess) ms[i].push_back(t);
      }
    }
    for (size_t i = 0; i < ok.size(); ++i) {
      if (ge[i]) cudaGraphExecDestroy(ge[i]);
      if (gr[i]) cudaGraphDestroy(gr[i]);
    }
    float best_t = 0.f;
    for (size_t i = 0; i < ok.size() && rc == CPM_OK; ++i) {
      if (ms[i].empty()) continue;
      std::sort(ms[i].begin(), ms[i].end());
      const float med = ms[i][ms[i].size() / 2];
      if (best_t == 0.f || med < best_t) {
        best_t = med;
        *best = ok[i];
      }
    }
  };
  // the S-apply kernel first, then the transform, then the charge assignment, then the z group
  // of the real-space pair kernels and the pair-kernel form, each stage with the choices so far
  Cfg best{keep_s, CPM_FFT_LIBRARY, CPM_MESH_SITES, keep_g, keep_p};
  {
    std::vector<Cfg> cand;
    for (int sv : {CPM_SAPPLY_ROWS, CPM_SAPPLY_STREAM, CPM_SAPPLY_STREAM16, CPM_SAPPLY_SYM, CPM_SAPPLY_SYM_TMA})
      cand.push_back({sv, best.fv, best.mv, best.gz, best.pv});
    choose(cand, &best);
  }
  if (rc == CPM_OK) choose({best, {best.sv, CPM_FFT_OWN, best.mv, best.gz, best.pv}}, &best);
  if (rc == CPM_OK) choose({best, {best.sv, best.fv, CPM_MESH_BRICK, best.gz, best.pv}}, &best);
  // the pair-kernel form and its z group together (the cell and third-law kernels prefer
  // different groups)
  if (rc == CPM_OK) {
    std::vector<Cfg> cand{best};
    for (int pv : {(int)CPM_PAIR_CELL, (int)CPM_PAIR_WARP_ELEC, (int)CPM_PAIR_WARP_ELYT, (int)CPM_PAIR_WARP,
                   (int)CPM_PAIR_N3_ELYT, (int)CPM_PAIR_N3_ELYT | (int)CPM_PAIR_WARP_ELEC})
      for (int gz : {1, 2, 3, 4})
        if ((pv != best.pv || gz != best.gz) && pair_group_ok(c, gz))
          cand.push_back({best.sv, best.fv, best.mv, gz, pv});
    choose(cand, &best);
  }
  if (rc != CPM_OK || !apply(best)) {
    c->pair_gz = keep_g;
    c->pair_variant = keep_p;
    c->sapply_variant = keep_s;
    c->fft_variant = keep_f;
    c->mesh_variant = keep_m;
  }
  cudaFree(f_scr);
  cudaFree(fe_scr);
  cudaFree(e_scr);
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  cudaStreamDestroy(cs);
  cudaFree(flush);
  if (choice_host) {
    choice_host[0] = c->sapply_variant;
    choice_host[1] = c->fft_variant;
    choice_host[2] = c->mesh_variant;
  }
  return rc;
}

extern "C" int cpm_profile_enable(cpm_ctx* c, int32_t capacity) {
  if (!c || capacity < 0) return CPM_ERR_ARG;
  if (c->prof_ev) {
    for (int k = 0; k < 2 * c->prof_cap; ++k) cudaEventDestroy(c->prof_ev[k]);
    delete[] c->prof_ev;
    delete[] c->prof_phase;
    c->prof_ev = nullptr;
    c->prof_phase = nullptr;
  }
  c->prof_cap = 0;
  c->prof_used = 0;
  if (capacity == 0) return CPM_OK;
  c->prof_ev = new cudaEvent_t[2 * (size_t)capacity];
  c->prof_phase = new int[capacity];
  for (int k = 0; k < 2 * capacity; ++k) CPM_CUDA(cudaEventCreate(&c->prof_ev[k]));
  c->prof_cap = capacity;
  return CPM_OK;
}

extern "C" int cpm_profile_read(cpm_ctx* c, double* ms, int64_t* count) {
  if (!c || !ms || !count) return CPM_ERR_ARG;
  for (int p = 0; p < CPM_NPHASES; ++p) {
    ms[p] = 0.0;
    count[p] = 0;
  }
  CPM_CUDA(cudaDeviceSynchronize());
  for (int k = 0; k < c->prof_used; ++k) {
    float t = 0.f;
    CPM_CUDA(cudaEventElapsedTime(&t, c->prof_ev[2 * k], c->prof_ev[2 * k + 1]));
    ms[c->prof_phase[k]] += t;
    count[c->prof_phase[k]] += 1;
  }
  c->prof_used = 0;
  return CPM_OK;
}

extern "C" int cpm_counters(const cpm_ctx* c, int64_t* kernel_launches) {
  if (!c || !kernel_launches) return CPM_ERR_ARG;
  *kernel_launches = c->launches;
  return CPM_OK;
}

// ------------------------------------------------------------------------------------------
// allocation-free single-replica charge update (cpm_step_charges_static)
// ------------------------------------------------------------------------------------------
// Scratch for cpm_step_charges_static, held by every device that loads the library.
static __device__ __align__(256) unsigned char g_cpm_static_scratch[CPM_STATIC_SCRATCH_BYTES];

namespace {
std::mutex g_static_mu;
constexpr int kMaxDevices = 64;
void* g_static_addr[kMaxDevices] = {};   // device address of the array, per device ordinal
}  // namespace

// Host code cannot use the array's name as a device address: its address on the current device is
// looked up with cudaGetSymbolAddress.  The lookup runs whenever a context is built on that device
// (refresh = true: a cudaDeviceReset invalidates every earlier context and may move the array, and
// a new build is the only way on), else on the first call on a device with no context built since
// the library was loaded.
static int static_scratch(void** out, bool refresh) {
  int dev = 0;
  CPM_CUDA(cudaGetDevice(&dev));
  if (dev < 0 || dev >= kMaxDevices) {
    cpm::set_error("device ordinal %d outside the supported range", dev);
    return CPM_ERR_ARG;
  }
  std::lock_guard<std::mutex> lock(g_static_mu);
  if (refresh || !g_static_addr[dev]) {
    void* p = nullptr;
    const cudaError_t e = cudaGetSymbolAddress(&p, g_cpm_static_scratch);
    if (e != cudaSuccess || !p) {
      g_static_addr[dev] = nullptr;
      cpm::set_error("cudaGetSymbolAddress(static scratch): %s", cudaGetErrorString(e));
      return CPM_ERR_CUDA;
    }
    g_static_addr[dev] = p;
  }
  *out = g_static_addr[dev];
  return CPM_OK;
}

// Set-up at context build (current device = the context's device).
int cpm_internal_static_scratch_setup() {
  void* p = nullptr;
  return static_scratch(&p, true);
}

extern "C" int cpm_step_charges_static(cpm_ctx* ctx, const int32_t* off, const double* xyzq, const double* dpsi,
                                       double* q, double* b, double* psibar, void* stream) {
  if (!ctx || !off || !xyzq || !dpsi || !q) {
    cpm::set_error("cpm_step_charges_static: null context or required pointer");
    return CPM_ERR_ARG;
  }
  if (reinterpret_cast<uintptr_t>(xyzq) % 32 != 0) {
    cpm::set_error("elyt_xyzq_dev must be 32-byte aligned");
    return CPM_ERR_ARG;
  }
  void* base_v = nullptr;
  CPM_TRY(static_scratch(&base_v, false));
  unsigned char* base = static_cast<unsigned char*>(base_v);
  const size_t tsz = ctx->mixed ? sizeof(float) : sizeof(double);
  const size_t v4 = ctx->mixed ? sizeof(float4) : sizeof(double4_32a);
  const size_t cap = ctx->p.max_elyt, ncell = ctx->ncell;
  const size_t sizes[] = {tsz * ctx->Mr_s,          tsz * ctx->Mr_s,             2 * tsz * ctx->Mc_s,
                          sizeof(int) * cap,        sizeof(int) * ncell,         sizeof(int) * (ncell + 1),
                          sizeof(int) * cap,        v4 * cap,                    0 /* unused slot */,
                          sizeof(double) * ctx->ne, sizeof(double) * ctx->ldb,   sizeof(float) * 2 * ctx->ldx,
                          sizeof(double) * cpm::NSCAL, v4 * cap,                 tsz * ctx->ne,
                          sizeof(double) * 2 * ctx->ldh, sizeof(double) * 2 * ctx->nh};
  constexpr int NREG = sizeof(sizes) / sizeof(sizes[0]);
  size_t offs[NREG], total = 0;
  for (int k = 0; k < NREG; ++k) {
    offs[k] = total;
    total += (sizes[k] + 255) & ~size_t(255);
  }
  if (total > CPM_STATIC_SCRATCH_BYTES) {
    cpm::set_error("cpm_step_charges_static: this context needs %zu bytes of scratch, the static array holds %u",
                   total, CPM_STATIC_SCRATCH_BYTES);
    return CPM_ERR_CAPACITY;
  }
  // Shallow copy: S, stencils, tables, plans and the status word are shared read-only; every
  // per-call workspace points into the static array.  One replica, single-batch FFT plan, no
  // profiling.
  cpm_ctx t = *ctx;
  t.p.max_replicas = 1;
  t.have_plan[1] = false;
  t.prof_cap = t.prof_used = 0;
  t.prof_ev = nullptr;
  t.prof_phase = nullptr;
  t.mesh_r = base + offs[0];
  t.mesh_phi = base + offs[1];
  t.mesh_c = base + offs[2];
  t.l_cell = reinterpret_cast<int*>(base + offs[3]);
  t.l_count = reinterpret_cast<int*>(base + offs[4]);
  t.l_start = reinterpret_cast<int*>(base + offs[5]);
  t.l_sorted = reinterpret_cast<int*>(base + offs[6]);
  t.l_loc32 = ctx->mixed ? reinterpret_cast<float4*>(base + offs[7]) : nullptr;
  t.l_loc64 = ctx->mixed ? nullptr : reinterpret_cast<double4_32a*>(base + offs[7]);
  t.phi_real = reinterpret_cast<double*>(base + offs[9]);
  t.b_tmp = reinterpret_cast<double*>(base + offs[10]);
  t.b32 = reinterpret_cast<float*>(base + offs[11]);
  t.scal = reinterpret_cast<double*>(base + offs[12]);
  t.l_tmp = base + offs[13];
  t.qT = base + offs[14];
  t.qpart = nullptr;                    // the streaming S-apply's partial sums live in the context
  t.brick_ok = false;                   // so does the padded mesh of the brick charge assignment
  t.sym_ok = false;                     // and the partial sums of the packed S-apply
  t.ypm = ctx->mirror ? reinterpret_cast<double*>(base + offs[15]) : nullptr;
  t.qpm = ctx->mirror ? reinterpret_cast<double*>(base + offs[16]) : nullptr;
  cudaStream_t st = (cudaStream_t)stream;
  // The array keeps the previous call's contents: the S-apply reads the padding of b up to the
  // row stride, so that must be zero.  (The counts, mesh and reduction slots are cleared by the
  // step itself.)
  CPM_CUDA(cudaMemsetAsync(t.b_tmp, 0, sizes[10], st));
  CPM_CUDA(cudaMemsetAsync(t.b32, 0, sizes[11], st));
  if (ctx->mirror) CPM_CUDA(cudaMemsetAsync(t.ypm, 0, sizes[15], st));
  const int s = ctx->mixed
                    ? cpm::run<float>(&t, 1, off, xyzq, dpsi, true, q, b, psibar, nullptr, nullptr, nullptr, st)
                    : cpm::run<double>(&t, 1, off, xyzq, dpsi, true, q, b, psibar, nullptr, nullptr, nullptr, st);
  ctx->launches = t.launches;
  return s;
}
