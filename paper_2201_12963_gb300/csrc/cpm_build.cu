// Build of the constant-potential context: elastance A (Eq. 3) in float64 on the GPU, its
// Cholesky factorisation and inverse, the projected inverse S = O A^-1 (Eqs. 8-9) or
// O_1 O A^-1 (Eqs. 13-15), S v, the fixed electrode B-spline stencils, the SPME influence
// function and every workspace the per-step calls use.  Also: status, info and teardown.
#include "cpm_internal.cuh"

#include <algorithm>
#include <unordered_map>
#include <cstdarg>
#include <cstring>
#include <vector>

namespace cpm {

static thread_local std::string g_last_error;

void set_error(const char* fmt, ...) {
  char buf[1024];
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(buf, sizeof(buf), fmt, ap);
  va_end(ap);
  g_last_error = buf;
}

// ------------------------------------------------------------------------------------------
// A: real-space Gaussian-Gaussian part over every periodic image within rcut (float64).
//   A_ij = KE sum_n (erfc(alpha r) - erfc(eta r / sqrt 2)) / r,  r = |r_i - r_j + n L| < rcut,
//   excluding i == j at n = 0; plus the self term KE (sqrt2 eta - 2 alpha)/sqrt(pi) on the diagonal.
// Rows and columns may be different site sets (rows[i], cols[j]; same = 1 when they coincide, which
// enables the self exclusion and the self term); X[j * lda + i] = A(rows[i], cols[j]).
// ------------------------------------------------------------------------------------------
__global__ void k_build_areal(const double4_32a* __restrict__ rows, const double4_32a* __restrict__ cols, int n,
                              int lda, int same, double bx, double by, double bz,
                              const double3* __restrict__ shifts, int nshift, double alpha, double beta,
                              double rc2, double self_term, double* __restrict__ X) {
  const int j = blockIdx.x * blockDim.x + threadIdx.x;
  const int i = blockIdx.y * blockDim.y + threadIdx.y;
  if (i >= n || j >= n) return;
  const bool diag = same && i == j;
  const double4_32a a = rows[i], b = cols[j];
  double dx = a.x - b.x, dy = a.y - b.y, dz = a.z - b.z;
  dx -= bx * rint(dx / bx);
  dy -= by * rint(dy / by);
  dz -= bz * rint(dz / bz);
  double s = 0.0;
  for (int k = 0; k < nshift; ++k) {
    const double3 sh = shifts[k];
    const double x = dx + sh.x, y = dy + sh.y, z = dz + sh.z;
    const double r2 = x * x + y * y + z * z;
    if (r2 < rc2 && !(diag && sh.x == 0.0 && sh.y == 0.0 && sh.z == 0.0)) {
      const double r = sqrt(r2);
      s += (erfc(alpha * r) - erfc(beta * r)) / r;
    }
  }
  if (diag) s += self_term;
  X[(size_t)j * lda + i] = KE * s;
}

// ------------------------------------------------------------------------------------------
// A: reciprocal part through the SPME mesh operator, A_k = W^T Phi W: W_j is the B-spline
// stencil of site j (the fixed stencils of the per-step gather), Phi the mesh convolution with the
// influence function G of the per-step calls.  Column j of A_k is the mesh potential of a unit
// charge on site j gathered at every row site, so the matrix is exactly the discrete operator the
// per-step b, forces and energy use.  Float64 throughout; one mesh per column of a batch.
// ------------------------------------------------------------------------------------------
// mesh[b] = unit charge of site cols[b] spread with its stencil (the p^3 points are distinct since
// every K_d >= 2p); the meshes were cleared by the caller.
__global__ void k_unit_spread(const int* __restrict__ cols, int nb, const int4* __restrict__ base,
                              const double* __restrict__ th, int P, int K1, int K2, int K3, long long Mr_s,
                              double* __restrict__ mesh) {
  const int b = blockIdx.x;
  if (b >= nb) return;
  const int site = cols[b];
  const int4 bs = base[site];
  const double* w = th + (size_t)site * 3 * PMAX;
  double* m = mesh + (size_t)b * Mr_s;
  for (int t = threadIdx.x; t < P * P * P; t += blockDim.x) {
    const int tx = t / (P * P), ty = (t / P) % P, tz = t % P;
    const int gx = wrap_index(bs.x - tx, K1), gy = wrap_index(bs.y - ty, K2), gz = wrap_index(bs.z - tz, K3);
    m[((size_t)gx * K2 + gy) * K3 + gz] = w[tx] * w[PMAX + ty] * w[2 * PMAX + tz];
  }
}

__global__ void k_mul_g(double2* __restrict__ spec, const double* __restrict__ G, long long Mc, long long Mc_s,
                        int nb) {
  const int b = blockIdx.y;
  if (b >= nb) return;
  double2* c = spec + (size_t)b * Mc_s;
  for (long long k = blockIdx.x * (long long)blockDim.x + threadIdx.x; k < Mc; k += (long long)gridDim.x * blockDim.x) {
    const double g = G[k];
    double2 v = c[k];
    v.x *= g;
    v.y *= g;
    c[k] = v;
  }
}

// X_o[(col0 + b) * lda + r] += sum_g W_{rows_o[r]}(g) phi_b(g), one warp per (row, column b);
// grid.z selects the output (row set, matrix).
struct GatherOut {
  const int* rows[2];
  double* X[2];
};
__global__ void __launch_bounds__(256) k_gather_cols(GatherOut o, int nrows, int lda, int col0, int nb,
                                                     const int4* __restrict__ base, const double* __restrict__ th,
                                                     int P, int K1, int K2, int K3, long long Mr_s,
                                                     const double* __restrict__ phi) {
  const int b = blockIdx.y;
  const int lane = threadIdx.x & 31;
  const int r = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  if (b >= nb || r >= nrows) return;
  const int site = o.rows[blockIdx.z] ? o.rows[blockIdx.z][r] : r;
  const int4 bs = base[site];
  const double* w = th + (size_t)site * 3 * PMAX;
  const double* m = phi + (size_t)b * Mr_s;
  double acc = 0.0;
  for (int task = lane; task < P * P; task += 32) {
    const int ty = task / P, tz = task - ty * P;
    const int gy = wrap_index(bs.y - ty, K2), gz = wrap_index(bs.z - tz, K3);
    double s = 0.0;
    for (int tx = 0; tx < P; ++tx) s += w[tx] * m[((size_t)wrap_index(bs.x - tx, K1) * K2 + gy) * K3 + gz];
    acc += s * w[PMAX + ty] * w[2 * PMAX + tz];
  }
  acc = warp_sum(acc);
  if (lane == 0) o.X[blockIdx.z][(size_t)(col0 + b) * lda + r] += acc;
}

// Mirror blocks: (P, Q) -> (P + Q, P - Q) in place, n x n with leading dimension lda.
__global__ void k_plus_minus(double* __restrict__ Pm, double* __restrict__ Qm, int n, int lda) {
  const int j = blockIdx.x * blockDim.x + threadIdx.x;
  const int i = blockIdx.y * blockDim.y + threadIdx.y;
  if (i >= n || j >= n) return;
  const size_t k = (size_t)j * lda + i;
  const double a = Pm[k], b = Qm[k];
  Pm[k] = a + b;
  Qm[k] = a - b;
}

// Reciprocal-space factor table for one chunk of half-space k-vectors, column-major [ne x 2kc]:
// column 2c = sqrt(w_k) cos(k.r_i), column 2c+1 = sqrt(w_k) sin(k.r_i), so that
// T T^T = sum_k w_k cos(k.(r_i - r_j)) (the direct Ewald reciprocal sum).
__global__ void k_build_trig(const double4_32a* __restrict__ pos, int ne, const double4_32a* __restrict__ kv,
                             int kc, double* __restrict__ T) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  const int c = blockIdx.y;
  if (i >= ne || c >= kc) return;
  const double4_32a k = kv[c];   // (kx, ky, kz, sqrt(w))
  const double4_32a r = pos[i];
  double sn, cs;
  sincos(k.x * r.x + k.y * r.y + k.z * r.z, &sn, &cs);
  T[(size_t)(2 * c) * ne + i] = k.w * cs;
  T[(size_t)(2 * c + 1) * ne + i] = k.w * sn;
}

// Slab (Yeh-Berkowitz) term on the lower triangle: A_ij += KE (4 pi / V) z_i z_j.
__global__ void k_build_slab(const double* __restrict__ z, int ne, int lda, double coef, double* A) {
  const int j = blockIdx.x * blockDim.x + threadIdx.x;
  const int i = blockIdx.y * blockDim.y + threadIdx.y;
  if (i >= ne || j >= ne || i < j) return;
  A[(size_t)j * lda + i] += coef * z[i] * z[j];
}

// Copy the lower triangle (column-major) onto the upper one: X_ji = X_ij for i > j.
__global__ void k_symmetrize_lower(double* X, int n, int lda) {
  const int j = blockIdx.x * blockDim.x + threadIdx.x;
  const int i = blockIdx.y * blockDim.y + threadIdx.y;
  if (i >= n || j >= n || i <= j) return;
  X[(size_t)i * lda + j] = X[(size_t)j * lda + i];
}

// W[:,0] = A^-1 e, W[:,1] = A^-1 e_1 (row sums over all / sub-cell-1 columns), one warp per row.
__global__ void k_build_w(const double* __restrict__ Ainv, int n, int lda, const double* __restrict__ c1,
                          double* __restrict__ W) {
  const int warp = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int lane = threadIdx.x & 31;
  if (warp >= n) return;
  const double* row = Ainv + (size_t)warp * lda;
  double s0 = 0.0, s1 = 0.0;
  for (int j = lane; j < n; j += 32) {
    const double a = row[j];
    s0 += a;
    s1 += a * c1[j];
  }
  s0 = warp_sum(s0);
  s1 = warp_sum(s1);
  if (lane == 0) {
    W[2 * warp] = s0;
    W[2 * warp + 1] = s1;
  }
}

// S_ij = (A^-1)_ij - sum_ab W_ia M_ab W_jb  (in place).
__global__ void k_build_s(double* S, int n, int lda, const double* __restrict__ W, int ncons,
                          double m00, double m01, double m10, double m11) {
  const int j = blockIdx.x * blockDim.x + threadIdx.x;
  const int i = blockIdx.y * blockDim.y + threadIdx.y;
  if (i >= n || j >= n) return;
  const double wi0 = W[2 * i], wj0 = W[2 * j];
  double corr = wi0 * m00 * wj0;
  if (ncons == 2) {
    const double wi1 = W[2 * i + 1], wj1 = W[2 * j + 1];
    corr += wi0 * m01 * wj1 + wi1 * m10 * wj0 + wi1 * m11 * wj1;
  }
  S[(size_t)i * lda + j] -= corr;
}

// y = S x, one warp per row (float64).
__global__ void k_matvec64(const double* __restrict__ S, int n, int lda, const double* __restrict__ x,
                           double* __restrict__ y) {
  const int warp = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int lane = threadIdx.x & 31;
  if (warp >= n) return;
  const double* row = S + (size_t)warp * lda;
  double s = 0.0;
  for (int j = lane; j < n; j += 32) s += row[j] * x[j];
  s = warp_sum(s);
  if (lane == 0) y[warp] = s;
}

__global__ void k_to_float(const double* __restrict__ S, int n, int lda, float* __restrict__ D, int ldd) {
  const int j = blockIdx.x * blockDim.x + threadIdx.x;
  const int i = blockIdx.y;
  if (j >= ldd) return;
  D[(size_t)i * ldd + j] = (j < n) ? (float)S[(size_t)i * lda + j] : 0.0f;
}

// ------------------------------------------------------------------------------------------
// host helpers
// ------------------------------------------------------------------------------------------
// Cardinal B-spline weights (same recursion as the device helper, float64 on the host).
static void bspline_host(double f, int p, double* w, double* dw) {
  for (int t = 0; t < PMAX; ++t) w[t] = dw[t] = 0.0;
  w[0] = 1.0;
  for (int n = 2; n <= p; ++n) {
    if (n == p)
      for (int t = 0; t < n; ++t) dw[t] = w[t] - (t > 0 ? w[t - 1] : 0.0);
    for (int t = n - 1; t >= 0; --t) {
      const double a = (t < n - 1) ? w[t] : 0.0;
      const double b = (t > 0) ? w[t - 1] : 0.0;
      w[t] = ((f + t) * a + (n - f - t) * b) / (n - 1);
    }
  }
}

static double wrap_coord(double x, double L) {
  double y = x - L * std::floor(x / L);
  if (y >= L) y -= L;
  if (y < 0) y = 0;
  return y;
}

template <typename T> static int dev_alloc(T** p, size_t count) {
  if (count == 0) count = 1;
  cudaError_t e = cudaMalloc((void**)p, count * sizeof(T));
  if (e != cudaSuccess) {
    set_error("cudaMalloc(%zu bytes): %s", count * sizeof(T), cudaGetErrorString(e));
    *p = nullptr;
    return e == cudaErrorMemoryAllocation ? CPM_ERR_NOMEM : CPM_ERR_CUDA;
  }
  return CPM_OK;
}

template <typename T> static int upload(T** d, const std::vector<T>& h, cudaStream_t st) {
  CPM_TRY(dev_alloc(d, h.size()));
  CPM_CUDA(cudaMemcpyAsync(*d, h.data(), h.size() * sizeof(T), cudaMemcpyHostToDevice, st));
  return CPM_OK;
}

// True if two electrode sites lie within tol of each other (periodic images included).  A
// coincident pair makes the Gaussian-Gaussian kernel (erfc(alpha r) - erfc(eta r / sqrt 2)) / r
// of A a 0/0 and A singular.  Sites are wrapped into the box and hashed on cells of edge
// h >= 1e-3 A >> tol (at most 2^20 cells per axis), so a pair within tol shares a cell or sits in
// adjacent ones (the last cell of an axis is adjacent to the first).
static bool coincident_sites(const double box[3], int32_t ne, const double* xyz, double tol) {
  long long n[3];
  double h[3];
  for (int d = 0; d < 3; ++d) {
    h[d] = std::max(1e-3, box[d] / 1048576.0);
    n[d] = std::max(1LL, std::min(1048576LL, (long long)std::ceil(box[d] / h[d])));
  }
  std::vector<double> w(3 * (size_t)ne);
  std::vector<long long> cid(3 * (size_t)ne);
  for (int i = 0; i < ne; ++i)
    for (int d = 0; d < 3; ++d) {
      double x = std::fmod(xyz[3 * i + d], box[d]);
      if (x < 0) x += box[d];
      if (x >= box[d]) x -= box[d];
      w[3 * i + d] = x;
      cid[3 * i + d] = std::min((long long)(x / h[d]), n[d] - 1);
    }
  auto key = [&](long long a, long long b, long long c) {
    return ((uint64_t)a * (uint64_t)n[1] + (uint64_t)b) * (uint64_t)n[2] + (uint64_t)c;
  };
  std::unordered_map<uint64_t, std::vector<int>> grid;
  grid.reserve(2 * (size_t)ne);
  for (int i = 0; i < ne; ++i) {
    for (int da = -1; da <= 1; ++da)
      for (int db = -1; db <= 1; ++db)
        for (int dc = -1; dc <= 1; ++dc) {
          const long long a = (cid[3 * i] + da + n[0]) % n[0];
          const long long b = (cid[3 * i + 1] + db + n[1]) % n[1];
          const long long c = (cid[3 * i + 2] + dc + n[2]) % n[2];
          auto it = grid.find(key(a, b, c));
          if (it == grid.end()) continue;
          for (int j : it->second) {
            double r2 = 0;
            for (int d = 0; d < 3; ++d) {
              double dx = w[3 * i + d] - w[3 * j + d];
              dx -= box[d] * std::round(dx / box[d]);
              r2 += dx * dx;
            }
            if (r2 < tol * tol) return true;
          }
        }
    grid[key(cid[3 * i], cid[3 * i + 1], cid[3 * i + 2])].push_back(i);
  }
  return false;
}

static int validate(const cpm_params* p, int32_t ne, const double* xyz, const int32_t* side,
                    const int32_t* cell) {
  if (!p || !xyz || !side || ne < 2) return CPM_ERR_ARG;
  for (int d = 0; d < 3; ++d)
    if (!(p->box[d] > 0) || !std::isfinite(p->box[d]) || p->grid[d] < 2 * p->spme_order) return CPM_ERR_ARG;
  if (p->grid[2] % 2) return CPM_ERR_ARG;
  if (!(p->eta > 0) || !(p->alpha > 0) || !(p->alpha < p->eta / std::sqrt(2.0))) return CPM_ERR_ARG;
  if (!(p->rcut > 0)) return CPM_ERR_ARG;
  if (p->spme_order < 3 || p->spme_order > PMAX) return CPM_ERR_ARG;
  if (p->geometry < CPM_FF || p->geometry > CPM_SLAB) return CPM_ERR_ARG;
  if (p->precision != CPM_FP64 && p->precision != CPM_MIXED) return CPM_ERR_ARG;
  if (p->max_replicas < 1 || p->max_elyt < 1) return CPM_ERR_ARG;
  if (p->geometry == CPM_SLAB && !(p->slab_factor >= 1.0)) return CPM_ERR_ARG;
  if (p->geometry == CPM_DOUBLED && !cell) return CPM_ERR_ARG;
  if (p->matrix_kspace != CPM_KSPACE_EWALD && p->matrix_kspace != CPM_KSPACE_MESH) return CPM_ERR_ARG;
  if (p->dc_blocks < CPM_DC_AUTO || p->dc_blocks > CPM_DC_FULL) return CPM_ERR_ARG;
  for (int i = 0; i < ne; ++i) {
    if (side[i] != 1 && side[i] != -1) return CPM_ERR_ARG;
    if (p->geometry == CPM_DOUBLED && cell[i] != 0 && cell[i] != 1) return CPM_ERR_ARG;
    for (int d = 0; d < 3; ++d)
      if (!std::isfinite(xyz[3 * i + d])) return CPM_ERR_NONFINITE;
  }
  if (coincident_sites(p->box, ne, xyz, 1e-6)) return CPM_ERR_ARG;
  return CPM_OK;
}

// Influence function on the half spectrum [K1][K2][K3/2+1], incl. KE:
//   G(m) = KE (4 pi / V) exp(-k^2 / 4 alpha^2) / k^2 * prod_d 1 / |sum_{t=0}^{p-2} M_p(t+1) e^{2 pi i m_d t / K_d}|^2
// (Essmann et al. 1995); G(0) = 0, and G = 0 where an odd order's denominator vanishes (Nyquist).
static void influence_host(const cpm_ctx* c, std::vector<double>& G) {
  const int K1 = c->K[0], K2 = c->K[1], K3 = c->K[2], p = c->P;
  double w[PMAX], dw[PMAX];
  bspline_host(0.0, p, w, dw);   // w[t] = M_p(t)
  std::vector<double> den[3];
  for (int d = 0; d < 3; ++d) {
    const int K = c->K[d];
    den[d].resize(K);
    for (int n = 0; n < K; ++n) {
      double re = 0, im = 0;
      for (int t = 0; t <= p - 2; ++t) {
        const double ph = 2.0 * PI * n * t / K;
        re += w[t + 1] * std::cos(ph);
        im += w[t + 1] * std::sin(ph);
      }
      den[d][n] = re * re + im * im;
    }
  }
  const int K3h = K3 / 2 + 1;
  G.assign((size_t)K1 * K2 * K3h, 0.0);
  const double a2 = c->p.alpha * c->p.alpha;
  for (int n1 = 0; n1 < K1; ++n1) {
    const int m1 = n1 <= K1 / 2 ? n1 : n1 - K1;
    for (int n2 = 0; n2 < K2; ++n2) {
      const int m2 = n2 <= K2 / 2 ? n2 : n2 - K2;
      for (int n3 = 0; n3 < K3h; ++n3) {
        const int m3 = n3;
        if (m1 == 0 && m2 == 0 && m3 == 0) continue;
        const double d = den[0][n1] * den[1][n2] * den[2][n3];
        if (den[0][n1] < 1e-10 || den[1][n2] < 1e-10 || den[2][n3] < 1e-10) continue;
        const double kx = 2.0 * PI * m1 / c->ebox[0], ky = 2.0 * PI * m2 / c->ebox[1],
                     kz = 2.0 * PI * m3 / c->ebox[2];
        const double k2 = kx * kx + ky * ky + kz * kz;
        G[((size_t)n1 * K2 + n2) * K3h + n3] = KE * 4.0 * PI / c->V * std::exp(-k2 / (4.0 * a2)) / k2 / d;
      }
    }
  }
}

static int make_plans(cpm_ctx* c) {
  int n[3] = {c->K[0], c->K[1], c->K[2]};
  const int batches[2] = {1, c->p.max_replicas};
  for (int b = 0; b < 2; ++b) {
    if (b == 1 && batches[1] == 1) break;
    const cufftType tf = c->mixed ? CUFFT_R2C : CUFFT_D2Z;
    const cufftType tb = c->mixed ? CUFFT_C2R : CUFFT_Z2D;
    int nr[3] = {n[0], n[1], n[2]};
    int nh[3] = {n[0], n[1], n[2] / 2 + 1};
    CPM_LIB(cufftPlanMany(&c->plan_r2c[b], 3, n, nr, 1, (int)c->Mr_s, nh, 1, (int)c->Mc_s, tf,
                          batches[b]) == CUFFT_SUCCESS, "cufftPlanMany(r2c)");
    CPM_LIB(cufftPlanMany(&c->plan_c2r[b], 3, n, nh, 1, (int)c->Mc_s, nr, 1, (int)c->Mr_s, tb,
                          batches[b]) == CUFFT_SUCCESS, "cufftPlanMany(c2r)");
    c->have_plan[b] = true;
  }
  return CPM_OK;
}

// Cholesky factorisation and inverse of the SPD matrix X (n x n, lower triangle, lda) in place,
// then the upper triangle is filled from the lower one.
static int cholesky_inverse(cpm_ctx* c, double* X, int n, int lda, const char* what, cudaStream_t st) {
  int lwork = 0, lwork2 = 0;
  CPM_LIB(cusolverDnDpotrf_bufferSize(c->solver, CUBLAS_FILL_MODE_LOWER, n, X, lda, &lwork) ==
              CUSOLVER_STATUS_SUCCESS, "potrf_bufferSize");
  CPM_LIB(cusolverDnDpotri_bufferSize(c->solver, CUBLAS_FILL_MODE_LOWER, n, X, lda, &lwork2) ==
              CUSOLVER_STATUS_SUCCESS, "potri_bufferSize");
  lwork = std::max(lwork, lwork2);
  double* work = nullptr;
  int* dinfo = nullptr;
  CPM_TRY(dev_alloc(&work, (size_t)lwork));
  CPM_TRY(dev_alloc(&dinfo, 1));
  int info = 0;
  CPM_LIB(cusolverDnDpotrf(c->solver, CUBLAS_FILL_MODE_LOWER, n, X, lda, work, lwork, dinfo) ==
              CUSOLVER_STATUS_SUCCESS, "cusolverDnDpotrf");
  CPM_CUDA(cudaMemcpyAsync(&info, dinfo, sizeof(int), cudaMemcpyDeviceToHost, st));
  CPM_CUDA(cudaStreamSynchronize(st));
  if (info != 0) {
    cudaFree(work);
    cudaFree(dinfo);
    set_error("Cholesky factorisation of %s failed at column %d (not positive definite)", what, info);
    return CPM_ERR_NOT_SPD;
  }
  CPM_LIB(cusolverDnDpotri(c->solver, CUBLAS_FILL_MODE_LOWER, n, X, lda, work, lwork, dinfo) ==
              CUSOLVER_STATUS_SUCCESS, "cusolverDnDpotri");
  CPM_CUDA(cudaMemcpyAsync(&info, dinfo, sizeof(int), cudaMemcpyDeviceToHost, st));
  CPM_CUDA(cudaStreamSynchronize(st));
  cudaFree(work);
  cudaFree(dinfo);
  if (info != 0) {
    set_error("inverse of the Cholesky factor of %s failed (info %d)", what, info);
    return CPM_ERR_NOT_SPD;
  }
  dim3 blk(32, 8), grd((n + 31) / 32, (n + 7) / 8);
  k_symmetrize_lower<<<grd, blk, 0, st>>>(X, n, lda);
  CPM_LAUNCH();
  return CPM_OK;
}

// Periodic image shifts within rcut (a box edge shorter than 2 rcut needs more than one image).
static std::vector<double3> image_shifts(const cpm_ctx* c) {
  std::vector<double3> shifts;
  int nmax[3];
  for (int d = 0; d < 3; ++d) nmax[d] = (int)std::floor(c->p.rcut / c->ebox[d] + 0.5);
  for (int a = -nmax[0]; a <= nmax[0]; ++a)
    for (int b = -nmax[1]; b <= nmax[1]; ++b)
      for (int g = -nmax[2]; g <= nmax[2]; ++g)
        shifts.push_back(make_double3(a * c->ebox[0], b * c->ebox[1], g * c->ebox[2]));
  return shifts;
}

// X(rows, cols) += KE real-space Gaussian-Gaussian sums (+ self terms when same).
static int real_space_block(cpm_ctx* c, const double4_32a* rows, const double4_32a* cols, int n, int lda, int same,
                            double* X, cudaStream_t st) {
  const std::vector<double3> shifts = image_shifts(c);
  double3* dsh = nullptr;
  CPM_TRY(upload(&dsh, shifts, st));
  const double self = (std::sqrt(2.0) * c->p.eta - 2.0 * c->p.alpha) / std::sqrt(PI);
  dim3 blk(32, 8), grd((n + 31) / 32, (n + 7) / 8);
  k_build_areal<<<grd, blk, 0, st>>>(rows, cols, n, lda, same, c->ebox[0], c->ebox[1], c->ebox[2], dsh,
                                     (int)shifts.size(), c->p.alpha, c->p.eta / std::sqrt(2.0),
                                     c->p.rcut * c->p.rcut, self, X);
  CPM_LAUNCH();
  CPM_CUDA(cudaStreamSynchronize(st));
  cudaFree(dsh);
  return CPM_OK;
}

// Half-space k-vectors of the direct Ewald sum, (kx, ky, kz, sqrt(w_k)) with
// w_k = 2 KE (4 pi / V) exp(-k^2 / 4 alpha^2) / k^2.
static std::vector<double4_32a> ewald_kvectors(const cpm_ctx* c) {
  const cpm_params& p = c->p;
  const double kmax = p.kmax_build > 0 ? p.kmax_build : 2.0 * p.alpha * std::sqrt(27.6);
  int mmax[3];
  for (int d = 0; d < 3; ++d) mmax[d] = (int)std::floor(kmax * c->ebox[d] / (2.0 * PI));
  std::vector<double4_32a> kv;
  for (int a = -mmax[0]; a <= mmax[0]; ++a)
    for (int b = -mmax[1]; b <= mmax[1]; ++b)
      for (int g = -mmax[2]; g <= mmax[2]; ++g) {
        const bool half = a > 0 || (a == 0 && b > 0) || (a == 0 && b == 0 && g > 0);
        if (!half) continue;
        const double kx = 2 * PI * a / c->ebox[0], ky = 2 * PI * b / c->ebox[1], kz = 2 * PI * g / c->ebox[2];
        const double k2 = kx * kx + ky * ky + kz * kz;
        if (k2 > kmax * kmax) continue;
        const double wk = 2.0 * 4.0 * PI / c->V * std::exp(-k2 / (4.0 * p.alpha * p.alpha)) / k2 * KE;
        kv.push_back(make_double4_32a(kx, ky, kz, std::sqrt(wk)));
      }
  return kv;
}

// Direct Ewald reciprocal sum: X += T_r T_c^T with T_s = [sqrt(w) cos(k.r), sqrt(w) sin(k.r)].
// rows == cols: DSYRK on the lower triangle; otherwise a full DGEMM.
static int ewald_kspace_block(cpm_ctx* c, const double4_32a* rows, const double4_32a* cols, int n, int lda,
                              double* X, cudaStream_t st) {
  const std::vector<double4_32a> kv = ewald_kvectors(c);
  if (kv.empty()) return CPM_OK;
  const int kc = 2048;
  double4_32a* dkv = nullptr;
  double *Tr = nullptr, *Tc = nullptr;
  CPM_TRY(upload(&dkv, kv, st));
  CPM_TRY(dev_alloc(&Tc, (size_t)n * 2 * kc));
  if (rows != cols) CPM_TRY(dev_alloc(&Tr, (size_t)n * 2 * kc));
  const double one = 1.0;
  for (size_t k0 = 0; k0 < kv.size(); k0 += kc) {
    const int m = (int)std::min<size_t>(kc, kv.size() - k0);
    k_build_trig<<<dim3((n + 127) / 128, m), 128, 0, st>>>(cols, n, dkv + k0, m, Tc);
    CPM_LAUNCH();
    if (rows == cols) {
      CPM_LIB(cublasDsyrk(c->cublas, CUBLAS_FILL_MODE_LOWER, CUBLAS_OP_N, n, 2 * m, &one, Tc, n, &one, X, lda) ==
                  CUBLAS_STATUS_SUCCESS, "cublasDsyrk");
    } else {
      k_build_trig<<<dim3((n + 127) / 128, m), 128, 0, st>>>(rows, n, dkv + k0, m, Tr);
      CPM_LAUNCH();
      CPM_LIB(cublasDgemm(c->cublas, CUBLAS_OP_N, CUBLAS_OP_T, n, n, 2 * m, &one, Tr, n, Tc, n, &one, X, lda) ==
                  CUBLAS_STATUS_SUCCESS, "cublasDgemm");
    }
  }
  CPM_CUDA(cudaStreamSynchronize(st));
  cudaFree(Tr);
  cudaFree(Tc);
  cudaFree(dkv);
  return CPM_OK;
}

// Mesh form of the reciprocal part: for every column site cols[j] (device, ncols of them) and each
// output o < nout, X_o[j * lda + r] += (W^T Phi W)(rows_o[r], cols[j]) for r < nrows (rows_o = nullptr:
// r itself).  Columns go through the FFTs in batches.
static int mesh_kspace(cpm_ctx* c, const int* cols, int ncols, GatherOut o, int nout, int nrows, int lda,
                       cudaStream_t st) {
  const size_t per_col = sizeof(double) * c->Mr_s + sizeof(double2) * c->Mc_s;
  int B = (int)std::max<size_t>(1, std::min<size_t>(((size_t)2 << 30) / per_col, 64));
  B = std::min(B, ncols);
  double* mesh = nullptr;
  double2* spec = nullptr;
  CPM_TRY(dev_alloc(&mesh, (size_t)B * c->Mr_s));
  CPM_TRY(dev_alloc(&spec, (size_t)B * c->Mc_s));
  int n[3] = {c->K[0], c->K[1], c->K[2]};
  int nr[3] = {n[0], n[1], n[2]};
  int nh[3] = {n[0], n[1], n[2] / 2 + 1};
  cufftHandle fwd = 0, inv = 0;
  CPM_LIB(cufftPlanMany(&fwd, 3, n, nr, 1, (int)c->Mr_s, nh, 1, (int)c->Mc_s, CUFFT_D2Z, B) == CUFFT_SUCCESS,
          "cufftPlanMany(d2z, build)");
  CPM_LIB(cufftPlanMany(&inv, 3, n, nh, 1, (int)c->Mc_s, nr, 1, (int)c->Mr_s, CUFFT_Z2D, B) == CUFFT_SUCCESS,
          "cufftPlanMany(z2d, build)");
  CPM_LIB(cufftSetStream(fwd, st) == CUFFT_SUCCESS, "cufftSetStream");
  CPM_LIB(cufftSetStream(inv, st) == CUFFT_SUCCESS, "cufftSetStream");
  const int gblocks = (int)std::min<long long>((c->Mc + 255) / 256, 152 * 8);
  int rc = CPM_OK;
  for (int c0 = 0; c0 < ncols && rc == CPM_OK; c0 += B) {
    const int nb = std::min(B, ncols - c0);
    CPM_CUDA(cudaMemsetAsync(mesh, 0, sizeof(double) * (size_t)B * c->Mr_s, st));
    k_unit_spread<<<nb, 128, 0, st>>>(cols + c0, nb, c->e_base, c->e_th64, c->P, c->K[0], c->K[1], c->K[2], c->Mr_s,
                                      mesh);
    CPM_LAUNCH();
    if (cufftExecD2Z(fwd, mesh, (cufftDoubleComplex*)spec) != CUFFT_SUCCESS) rc = CPM_ERR_LIBRARY;
    k_mul_g<<<dim3(gblocks, nb), 256, 0, st>>>(spec, c->G64, c->Mc, c->Mc_s, nb);
    CPM_LAUNCH();
    if (cufftExecZ2D(inv, (cufftDoubleComplex*)spec, mesh) != CUFFT_SUCCESS) rc = CPM_ERR_LIBRARY;
    k_gather_cols<<<dim3((nrows * 32 + 255) / 256, nb, nout), 256, 0, st>>>(o, nrows, lda, c0, nb, c->e_base,
                                                                           c->e_th64, c->P, c->K[0], c->K[1],
                                                                           c->K[2], c->Mr_s, mesh);
    CPM_LAUNCH();
  }
  CPM_CUDA(cudaStreamSynchronize(st));
  cufftDestroy(fwd);
  cufftDestroy(inv);
  cudaFree(mesh);
  cudaFree(spec);
  if (rc != CPM_OK) set_error("cuFFT execution failed while building the mesh part of A");
  return rc;
}

static int kspace_block(cpm_ctx* c, const double4_32a* rows_pos, const double4_32a* cols_pos, const int* rows_idx,
                        const int* cols_idx, int n, int lda, double* X, cudaStream_t st) {
  if (c->p.matrix_kspace == CPM_KSPACE_MESH) {
    GatherOut o{{rows_idx, nullptr}, {X, nullptr}};
    return mesh_kspace(c, cols_idx, n, o, 1, n, lda, st);
  }
  return ewald_kspace_block(c, rows_pos, cols_pos, n, lda, X, st);
}

// Full matrix: A (ne x ne) -> S = A^-1 - A^-1 C (C^T A^-1 C)^-1 C^T A^-1, A^-1 C, S v.
static int finish_s32(cpm_ctx* c, int rows, cudaStream_t st);

static int build_full(cpm_ctx* c, const std::vector<double>& v, const std::vector<double>& c1,
                      const int32_t* side, cudaStream_t st) {
  const int ne = c->ne;
  const cpm_params& p = c->p;
  c->ld64 = c->ld32 = c->ldx = (ne + 3) & ~3;
  CPM_TRY(dev_alloc(&c->S64, (size_t)ne * c->ld64));
  double* A = c->S64;
  CPM_CUDA(cudaMemsetAsync(A, 0, sizeof(double) * (size_t)ne * c->ld64, st));
  CPM_TRY(real_space_block(c, c->e_pos64, c->e_pos64, ne, c->ld64, 1, A, st));
  {
    std::vector<int> iota(ne);
    for (int i = 0; i < ne; ++i) iota[i] = i;
    int* d_iota = nullptr;
    CPM_TRY(upload(&d_iota, iota, st));
    const int r = kspace_block(c, c->e_pos64, c->e_pos64, nullptr, d_iota, ne, c->ld64, A, st);
    cudaFree(d_iota);
    CPM_TRY(r);
  }
  if (p.geometry == CPM_SLAB) {
    dim3 blk(32, 8), grd((ne + 31) / 32, (ne + 7) / 8);
    k_build_slab<<<grd, blk, 0, st>>>(c->e_z, ne, c->ld64, KE * 4.0 * PI / c->V, A);
    CPM_LAUNCH();
  }
  CPM_TRY(cholesky_inverse(c, A, ne, c->ld64, "A", st));
  // ---------------- projection pieces ----------------
  CPM_TRY(dev_alloc(&c->W, (size_t)ne * 2));
  k_build_w<<<(ne * 32 + 255) / 256, 256, 0, st>>>(A, ne, c->ld64, c->e_c1, c->W);
  CPM_LAUNCH();
  std::vector<double> Wh((size_t)ne * 2);
  CPM_CUDA(cudaMemcpyAsync(Wh.data(), c->W, sizeof(double) * ne * 2, cudaMemcpyDeviceToHost, st));
  CPM_CUDA(cudaStreamSynchronize(st));
  // C^T W (ncons x ncons) and its inverse M
  double ctw[4] = {0, 0, 0, 0};
  for (int i = 0; i < ne; ++i) {
    ctw[0] += Wh[2 * i];                   // e^T A^-1 e
    ctw[1] += Wh[2 * i + 1];               // e^T A^-1 e_1
    ctw[2] += c1[i] * Wh[2 * i];           // e_1^T A^-1 e
    ctw[3] += c1[i] * Wh[2 * i + 1];       // e_1^T A^-1 e_1
    c->WTv[0] += Wh[2 * i] * v[i];
    c->WTv[1] += Wh[2 * i + 1] * v[i];
  }
  if (c->ncons == 1) {
    if (!(ctw[0] > 0)) { set_error("e^T A^-1 e is not positive"); return CPM_ERR_NOT_SPD; }
    c->Mh[0] = 1.0 / ctw[0];
  } else {
    const double det = ctw[0] * ctw[3] - ctw[1] * ctw[2];
    if (!(std::fabs(det) > 0)) { set_error("C^T A^-1 C is singular"); return CPM_ERR_NOT_SPD; }
    c->Mh[0] = ctw[3] / det;
    c->Mh[1] = -ctw[1] / det;
    c->Mh[2] = -ctw[2] / det;
    c->Mh[3] = ctw[0] / det;
  }
  {
    dim3 blk(32, 8), grd((ne + 31) / 32, (ne + 7) / 8);
    k_build_s<<<grd, blk, 0, st>>>(A, ne, c->ld64, c->W, c->ncons, c->Mh[0], c->Mh[1], c->Mh[2], c->Mh[3]);
    CPM_LAUNCH();
  }
  CPM_TRY(dev_alloc(&c->Sv, (size_t)ne));
  k_matvec64<<<(ne * 32 + 255) / 256, 256, 0, st>>>(c->S64, ne, c->ld64, c->e_v, c->Sv);
  CPM_LAUNCH();
  {
    std::vector<double> svh(ne);
    CPM_CUDA(cudaMemcpyAsync(svh.data(), c->Sv, sizeof(double) * ne, cudaMemcpyDeviceToHost, st));
    CPM_CUDA(cudaStreamSynchronize(st));
    c->dqdpsi = 0;
    for (int i = 0; i < ne; ++i)
      if (side[i] > 0) c->dqdpsi += svh[i];
  }
  return finish_s32(c, ne, st);
}

// Doubled cell whose sub-cell-1 electrode is the z-mirror image of the sub-cell-0 one: with the sites
// ordered (sub-cell 0 in index order, then their images), A = [[P, Q], [Q, P]], P = A(I0, I0),
// Q = A(I0, m(I0)).  With y+- = y_I0 +- y_m(I0) and the constraints e^T q = e_1^T q = 0 rewritten as
// 1^T q+ = 1^T q- = 0, the charges are q+- = S+- y+- with S+- the singly-constrained projected
// inverses of A+- = P +- Q, and q_I0 = (q+ + q-) / 2, q_m(I0) = (q+ - q-) / 2.  Two n x n
// factorisations replace one 2n x 2n one, and the S-apply streams half the bytes.
static int build_mirror(cpm_ctx* c, const std::vector<double4_32a>& pos, const std::vector<double>& v,
                        const int32_t* side, cudaStream_t st) {
  const int N = c->nh;
  const int ldh = (N + 3) & ~3;
  c->ldh = ldh;
  c->ld64 = c->ld32 = ldh;
  c->ldx = 2 * ldh;
  std::vector<double4_32a> pI(N), pJ(N);
  for (int k = 0; k < N; ++k) {
    pI[k] = pos[c->h_i0[k]];
    pJ[k] = pos[c->h_j[k]];
  }
  double4_32a *dI = nullptr, *dJ = nullptr;
  CPM_TRY(upload(&dI, pI, st));
  CPM_TRY(upload(&dJ, pJ, st));
  CPM_TRY(upload(&c->m_i0, c->h_i0, st));
  CPM_TRY(upload(&c->m_j, c->h_j, st));
  CPM_TRY(dev_alloc(&c->S64, (size_t)2 * N * ldh));
  double* Pm = c->S64;
  double* Qm = c->S64 + (size_t)N * ldh;
  CPM_CUDA(cudaMemsetAsync(c->S64, 0, sizeof(double) * (size_t)2 * N * ldh, st));
  CPM_TRY(real_space_block(c, dI, dI, N, ldh, 1, Pm, st));
  CPM_TRY(real_space_block(c, dJ, dI, N, ldh, 0, Qm, st));
  if (c->p.matrix_kspace == CPM_KSPACE_MESH) {
    GatherOut o{{c->m_i0, c->m_j}, {Pm, Qm}};
    CPM_TRY(mesh_kspace(c, c->m_i0, N, o, 2, N, ldh, st));
  } else {
    CPM_TRY(ewald_kspace_block(c, dI, dI, N, ldh, Pm, st));
    CPM_TRY(ewald_kspace_block(c, dJ, dI, N, ldh, Qm, st));
  }
  cudaFree(dI);
  cudaFree(dJ);
  {
    dim3 blk(32, 8), grd((N + 31) / 32, (N + 7) / 8);
    k_plus_minus<<<grd, blk, 0, st>>>(Pm, Qm, N, ldh);
    CPM_LAUNCH();
  }
  CPM_TRY(cholesky_inverse(c, Pm, N, ldh, "A+ = P + Q", st));
  CPM_TRY(cholesky_inverse(c, Qm, N, ldh, "A- = P - Q", st));
  // constraint indicator of the S-apply rows: zeros (A+ block), ones (A- block)
  std::vector<double> c1m(2 * (size_t)N, 0.0);
  for (int k = 0; k < N; ++k) c1m[N + k] = 1.0;
  CPM_TRY(upload(&c->e_c1m, c1m, st));
  // w+- = A+-^-1 1, M+- = 1 / 1^T w+-, S+- = A+-^-1 - w+- M+- w+-^T
  double* wtmp = nullptr;
  CPM_TRY(dev_alloc(&wtmp, (size_t)2 * N));
  std::vector<double> wpm[2];
  for (int blk = 0; blk < 2; ++blk) {
    double* X = blk ? Qm : Pm;
    k_build_w<<<(N * 32 + 255) / 256, 256, 0, st>>>(X, N, ldh, c->e_c1m, wtmp);   // e_c1m[0..N) = 0
    CPM_LAUNCH();
    std::vector<double> h(2 * (size_t)N);
    CPM_CUDA(cudaMemcpyAsync(h.data(), wtmp, sizeof(double) * 2 * N, cudaMemcpyDeviceToHost, st));
    CPM_CUDA(cudaStreamSynchronize(st));
    double sum = 0;
    wpm[blk].resize(N);
    for (int k = 0; k < N; ++k) {
      wpm[blk][k] = h[2 * k];
      sum += h[2 * k];
    }
    if (!(sum > 0)) {
      cudaFree(wtmp);
      set_error("1^T A%c^-1 1 is not positive", blk ? '-' : '+');
      return CPM_ERR_NOT_SPD;
    }
    c->Mh[blk] = 1.0 / sum;
    dim3 b2(32, 8), grd((N + 31) / 32, (N + 7) / 8);
    k_build_s<<<grd, b2, 0, st>>>(X, N, ldh, wtmp, 1, c->Mh[blk], 0.0, 0.0, 0.0);
    CPM_LAUNCH();
  }
  CPM_CUDA(cudaStreamSynchronize(st));
  cudaFree(wtmp);
  c->Mh[2] = c->Mh[3] = 0.0;
  // W in the S-apply epilogue's interleaved layout: rows of block + carry (w+, 0), rows of block - (0, w-)
  std::vector<double> Wint(4 * (size_t)N, 0.0), vpm(2 * (size_t)N);
  c->WTv[0] = c->WTv[1] = 0.0;
  for (int k = 0; k < N; ++k) {
    Wint[2 * k] = wpm[0][k];
    Wint[2 * (size_t)N + 2 * k + 1] = wpm[1][k];
    vpm[k] = v[c->h_i0[k]] + v[c->h_j[k]];
    vpm[N + k] = v[c->h_i0[k]] - v[c->h_j[k]];
    c->WTv[0] += wpm[0][k] * vpm[k];
    c->WTv[1] += wpm[1][k] * vpm[N + k];
  }
  CPM_TRY(upload(&c->W, Wint, st));
  double* dv = nullptr;
  CPM_TRY(upload(&dv, vpm, st));
  CPM_TRY(dev_alloc(&c->Sv, (size_t)2 * N));
  k_matvec64<<<(N * 32 + 255) / 256, 256, 0, st>>>(Pm, N, ldh, dv, c->Sv);
  CPM_LAUNCH();
  k_matvec64<<<(N * 32 + 255) / 256, 256, 0, st>>>(Qm, N, ldh, dv + N, c->Sv + N);
  CPM_LAUNCH();
  {
    std::vector<double> svh(2 * (size_t)N);
    CPM_CUDA(cudaMemcpyAsync(svh.data(), c->Sv, sizeof(double) * 2 * N, cudaMemcpyDeviceToHost, st));
    CPM_CUDA(cudaStreamSynchronize(st));
    c->dqdpsi = 0;
    for (int k = 0; k < N; ++k) {
      if (side[c->h_i0[k]] > 0) c->dqdpsi += 0.5 * (svh[k] + svh[N + k]);
      if (side[c->h_j[k]] > 0) c->dqdpsi += 0.5 * (svh[k] - svh[N + k]);
    }
  }
  cudaFree(dv);
  return finish_s32(c, 2 * N, st);
}

// Pairs every sub-cell-0 site with the sub-cell-1 site at its z-mirror image (x, y, L_z - z)
// (L_z the doubled length) within 1e-6 A; false if the electrode is not mirror-symmetric.
static bool find_mirror(cpm_ctx* c, const std::vector<double4_32a>& pos, const int32_t* cell) {
  const int ne = c->ne;
  int n0 = 0;
  for (int i = 0; i < ne; ++i) n0 += cell[i] == 0;
  if (2 * n0 != ne) return false;
  const double h = 1e-3, tol = 1e-6;
  long long nk[3];
  for (int d = 0; d < 3; ++d) nk[d] = std::max(1LL, (long long)std::ceil(c->ebox[d] / h));
  auto idx = [&](double x, int d) { return ((long long)std::floor(x / h) % nk[d] + nk[d]) % nk[d]; };
  auto key = [&](long long a, long long b, long long g) { return (a * nk[1] + b) * nk[2] + g; };
  std::unordered_map<long long, std::vector<int>> grid;
  for (int i = 0; i < ne; ++i)
    if (cell[i] == 1) grid[key(idx(pos[i].x, 0), idx(pos[i].y, 1), idx(pos[i].z, 2))].push_back(i);
  std::vector<char> used(ne, 0);
  c->h_i0.clear();
  c->h_j.clear();
  for (int i = 0; i < ne; ++i) {
    if (cell[i] != 0) continue;
    const double t[3] = {pos[i].x, pos[i].y, wrap_coord(c->ebox[2] - pos[i].z, c->ebox[2])};
    const long long k0[3] = {idx(t[0], 0), idx(t[1], 1), idx(t[2], 2)};
    int found = -1;
    for (int a = -1; a <= 1 && found < 0; ++a)
      for (int b = -1; b <= 1 && found < 0; ++b)
        for (int g = -1; g <= 1 && found < 0; ++g) {
          auto it = grid.find(key((k0[0] + a + nk[0]) % nk[0], (k0[1] + b + nk[1]) % nk[1], (k0[2] + g + nk[2]) % nk[2]));
          if (it == grid.end()) continue;
          for (int j : it->second) {
            if (used[j]) continue;
            const double r[3] = {pos[j].x, pos[j].y, pos[j].z};
            bool ok = true;
            for (int d = 0; d < 3 && ok; ++d) {
              double dd = r[d] - t[d];
              dd -= c->ebox[d] * std::rint(dd / c->ebox[d]);
              ok = std::fabs(dd) < tol;
            }
            if (ok) {
              found = j;
              break;
            }
          }
        }
    if (found < 0) return false;
    used[found] = 1;
    c->h_i0.push_back(i);
    c->h_j.push_back(found);
  }
  return true;
}

// ------------------------------------------------------------------------------------------
// matrix image: S (or the two mirror blocks), A^-1 C, S v and the projection scalars, so that a
// context can be rebuilt without assembling and factorising A (cpm_matrix_image and
// cpm_build_matrix_from_image).  The key is FNV-1a 64 (Fowler, Noll, Vo) over every input that
// determines A; an image is accepted only by a build whose inputs give the same key.
// ------------------------------------------------------------------------------------------
struct ImageHeader {
  char magic[8];                 // "CPMSIMG1"
  uint64_t key;
  int32_t ne, ncons, mirror, nh, ld64, reserved;
  int64_t nS, nW, nSv;           // float64 counts of the three arrays that follow the header
  double Mh[4], WTv[2], dqdpsi;
};
constexpr char kImageMagic[8] = {'C', 'P', 'M', 'S', 'I', 'M', 'G', '1'};

struct Fnv1a {
  uint64_t h = 1469598103934665603ull;
  void add(const void* data, size_t n) {
    const unsigned char* b = static_cast<const unsigned char*>(data);
    for (size_t i = 0; i < n; ++i) {
      h ^= b[i];
      h *= 1099511628211ull;
    }
  }
};

static uint64_t matrix_key(const cpm_params* p, int32_t ne, const double* xyz, const int32_t* side,
                           const int32_t* cell) {
  Fnv1a f;
  const int32_t version = 1;
  f.add(&version, sizeof version);
  f.add(p->box, sizeof p->box);
  f.add(&p->eta, sizeof(double));
  f.add(&p->alpha, sizeof(double));
  f.add(&p->rcut, sizeof(double));
  const double sf = p->geometry == CPM_SLAB ? p->slab_factor : 0.0;
  f.add(&sf, sizeof sf);
  const double km = p->matrix_kspace == CPM_KSPACE_EWALD ? p->kmax_build : 0.0;
  f.add(&km, sizeof km);
  f.add(&p->geometry, sizeof(int32_t));
  f.add(&p->matrix_kspace, sizeof(int32_t));
  const int32_t dcb = p->geometry == CPM_DOUBLED ? p->dc_blocks : 0;
  f.add(&dcb, sizeof dcb);
  if (p->matrix_kspace == CPM_KSPACE_MESH) {
    f.add(p->grid, sizeof p->grid);
    f.add(&p->spme_order, sizeof(int32_t));
  }
  f.add(&ne, sizeof ne);
  f.add(xyz, sizeof(double) * 3 * (size_t)ne);
  f.add(side, sizeof(int32_t) * (size_t)ne);
  if (p->geometry == CPM_DOUBLED && cell) f.add(cell, sizeof(int32_t) * (size_t)ne);
  return f.h;
}

// float32 copy of S for the mixed path (rows of the stored form: N_e, or 2 N_e/2 for mirror blocks)
static int finish_s32(cpm_ctx* c, int rows, cudaStream_t st) {
  if (!c->mixed) return CPM_OK;
  CPM_TRY(dev_alloc(&c->S32, (size_t)rows * c->ld32));
  k_to_float<<<dim3((c->ld32 + 255) / 256, rows), 256, 0, st>>>(c->S64, rows, c->ld64, c->S32, c->ld32);
  CPM_LAUNCH();
  return CPM_OK;
}

// Instead of build_full / build_mirror: the same device state from an image.
static int load_image(cpm_ctx* c, const void* image, int64_t bytes, uint64_t key, cudaStream_t st) {
  if (bytes < (int64_t)sizeof(ImageHeader)) {
    set_error("matrix image: %lld bytes is shorter than its header", (long long)bytes);
    return CPM_ERR_ARG;
  }
  ImageHeader h;
  std::memcpy(&h, image, sizeof h);
  const int ne = c->ne;
  const int rows = c->mirror ? 2 * c->nh : ne;
  const int ld = c->mirror ? ((c->nh + 3) & ~3) : ((ne + 3) & ~3);
  const int64_t nS = (int64_t)rows * ld, nW = c->mirror ? 4LL * c->nh : 2LL * ne, nSv = rows;
  if (std::memcmp(h.magic, kImageMagic, 8) != 0 || h.key != key || h.ne != ne || h.ncons != c->ncons ||
      h.mirror != (c->mirror ? 1 : 0) || h.nh != c->nh || h.ld64 != ld || h.nS != nS || h.nW != nW || h.nSv != nSv ||
      bytes != (int64_t)sizeof(ImageHeader) + 8 * (nS + nW + nSv)) {
    set_error("matrix image does not belong to these parameters and electrode (key or layout differs)");
    return CPM_ERR_ARG;
  }
  c->ld64 = c->ld32 = ld;
  if (c->mirror) {
    c->ldh = ld;
    c->ldx = 2 * ld;
    CPM_TRY(upload(&c->m_i0, c->h_i0, st));
    CPM_TRY(upload(&c->m_j, c->h_j, st));
    std::vector<double> c1m(2 * (size_t)c->nh, 0.0);
    for (int k = 0; k < c->nh; ++k) c1m[c->nh + k] = 1.0;
    CPM_TRY(upload(&c->e_c1m, c1m, st));
  } else {
    c->ldx = ld;
  }
  const double* src = reinterpret_cast<const double*>(static_cast<const char*>(image) + sizeof(ImageHeader));
  CPM_TRY(dev_alloc(&c->S64, (size_t)nS));
  CPM_TRY(dev_alloc(&c->W, (size_t)nW));
  CPM_TRY(dev_alloc(&c->Sv, (size_t)nSv));
  CPM_CUDA(cudaMemcpyAsync(c->S64, src, sizeof(double) * nS, cudaMemcpyHostToDevice, st));
  CPM_CUDA(cudaMemcpyAsync(c->W, src + nS, sizeof(double) * nW, cudaMemcpyHostToDevice, st));
  CPM_CUDA(cudaMemcpyAsync(c->Sv, src + nS + nW, sizeof(double) * nSv, cudaMemcpyHostToDevice, st));
  for (int k = 0; k < 4; ++k) c->Mh[k] = h.Mh[k];
  c->WTv[0] = h.WTv[0];
  c->WTv[1] = h.WTv[1];
  c->dqdpsi = h.dqdpsi;
  CPM_TRY(finish_s32(c, rows, st));
  CPM_CUDA(cudaStreamSynchronize(st));
  return CPM_OK;
}

// Electrode-electrode real-space force list (mixed precision): the electrode is frozen, so the
// Gaussian-Gaussian pair term of the electrode forces, F_i = KE q_i sum_j q_j G_ij with
// G_ij = [k(r) + 2/sqrt(pi) (alpha e^{-alpha^2 r^2} - beta e^{-beta^2 r^2})] d_ij / r^2,
// k(r) = (erfc(alpha r) - erfc(beta r)) / r, beta = eta / sqrt 2, d_ij = r_i - r_j (every periodic
// image within r_c, Sec. II.B), depends on the charges only through q_i q_j: G is evaluated once
// here in float64 and kept in float32, one CSR row per target in original order, entry
// (G_x, G_y, G_z, j).  The cell grid of the build (edge >= r_c / 2, stencil half-width sten)
// enumerates the images: an unwrapped neighbour cell index maps to a cell and an image shift.
static int build_ee_list(cpm_ctx* c, const std::vector<double4_32a>& pos, const std::vector<int4>& cc,
                         const std::vector<int>& start, const std::vector<int>& sorted, cudaStream_t st) {
  const int ne = c->ne;
  const double rc2 = c->p.rcut * c->p.rcut, alpha = c->p.alpha, beta = c->p.eta / std::sqrt(2.0);
  const double two_over_sqrt_pi = 2.0 / std::sqrt(M_PI);
  std::vector<int> ptr(ne + 1, 0);
  std::vector<float4> ent;
  ent.reserve((size_t)ne * 64);
  for (int i = 0; i < ne; ++i) {
    const int4 ci = cc[i];
    for (int dx = -c->sten[0]; dx <= c->sten[0]; ++dx)
      for (int dy = -c->sten[1]; dy <= c->sten[1]; ++dy)
        for (int dz = -c->sten[2]; dz <= c->sten[2]; ++dz) {
          const int u[3] = {ci.x + dx, ci.y + dy, ci.z + dz};
          int w[3];
          double sh[3];
          for (int d = 0; d < 3; ++d) {
            const int m = (int)std::floor((double)u[d] / c->nc[d]);
            w[d] = u[d] - m * c->nc[d];
            sh[d] = m * c->ebox[d];
          }
          const int cell = (w[0] * c->nc[1] + w[1]) * c->nc[2] + w[2];
          for (int k = start[cell]; k < start[cell + 1]; ++k) {
            const int j = sorted[k];
            const double ddx = pos[i].x - (pos[j].x + sh[0]), ddy = pos[i].y - (pos[j].y + sh[1]),
                         ddz = pos[i].z - (pos[j].z + sh[2]);
            const double r2 = ddx * ddx + ddy * ddy + ddz * ddz;
            if (r2 >= rc2 || r2 == 0.0) continue;      // (r = 0 only for i itself: coincident sites are refused)
            const double r = std::sqrt(r2);
            const double kr = (std::erfc(alpha * r) - std::erfc(beta * r)) / r;
            const double fr = (kr + two_over_sqrt_pi * (alpha * std::exp(-alpha * alpha * r2) -
                                                        beta * std::exp(-beta * beta * r2))) / r2;
            float4 e;
            e.x = (float)(fr * ddx);
            e.y = (float)(fr * ddy);
            e.z = (float)(fr * ddz);
            std::memcpy(&e.w, &j, sizeof(int));
            ent.push_back(e);
          }
        }
    ptr[i + 1] = (int)ent.size();
    if (ent.size() > (size_t)INT32_MAX - 4096) {
      set_error("electrode pair list above 2^31 entries");
      return CPM_ERR_ARG;
    }
  }
  if (ent.empty()) ent.push_back(make_float4(0.f, 0.f, 0.f, 0.f));   // never a null pointer
  c->ee_nnz = ptr[ne];
  // Compressed form: on a lattice electrode the pair vectors, hence the float32 G, repeat, and a
  // few hundred to a few thousand distinct values occur.  With at most 2^16 sites and fewer than
  // kEeTabMax distinct G (compared bit for bit, so both forms give the same products), an entry
  // becomes j | t << 16, t indexing a table of the distinct G: 4 bytes per pair instead of 16.
  if (ne <= 65536) {
    struct Key {
      uint32_t x, y, z;
      bool operator==(const Key& o) const { return x == o.x && y == o.y && z == o.z; }
    };
    struct KeyHash {
      size_t operator()(const Key& k) const {
        return (size_t)k.x * 0x9E3779B97F4A7C15ull ^ ((size_t)k.y * 0xC2B2AE3D27D4EB4Full + k.z);
      }
    };
    std::unordered_map<Key, int, KeyHash> seen;
    std::vector<float4> tab;
    // Rows padded to a multiple of 4 entries (the zero table entry, j = 0), so that the kernel
    // reads them as aligned 16-byte chunks: with `lpr` lanes per row, lane l takes chunks
    // l, l + lpr, l + 2 lpr, ...  Within a row the entries are sorted by j and placed so that the
    // lanes of one load instruction (the same chunk slot and the same entry of the chunk) hold
    // consecutive j: their charge gathers then fall on few cache sectors.
    int nsm = 0;
    CPM_CUDA(cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, c->dev));
    const int lpr = ((long long)ne * c->p.max_replicas * 8 < (long long)std::max(1, nsm) * 24 * 32) ? 32 : 8;
    std::vector<int> ptr4(ne + 1, 0);
    std::vector<unsigned> idx, rowv, slot;
    idx.reserve(ent.size() + 3 * (size_t)ne);
    const unsigned kPad = 0xFFFFFFFFu;         // placeholder until the zero entry's index is known
    bool fits = true;
    for (int i = 0; i < ne && fits; ++i) {
      rowv.clear();
      for (int k = ptr[i]; k < ptr[i + 1]; ++k) {
        Key key;
        std::memcpy(&key.x, &ent[k].x, 4);
        std::memcpy(&key.y, &ent[k].y, 4);
        std::memcpy(&key.z, &ent[k].z, 4);
        auto it = seen.find(key);
        int t;
        if (it == seen.end()) {
          t = (int)tab.size();
          if (t + 1 >= kEeTabMax) {        // one slot stays free for the zero entry
            fits = false;
            break;
          }
          seen.emplace(key, t);
          tab.push_back(make_float4(ent[k].x, ent[k].y, ent[k].z, 0.f));
        } else {
          t = it->second;
        }
        int j;
        std::memcpy(&j, &ent[k].w, sizeof(int));
        rowv.push_back((unsigned)j | ((unsigned)t << 16));
      }
      std::stable_sort(rowv.begin(), rowv.end(),
                       [](unsigned a, unsigned b) { return (a & 0xffffu) < (b & 0xffffu); });
      while (rowv.size() % 4) rowv.push_back(kPad);
      const int nch = (int)rowv.size() / 4;
      slot.clear();                            // positions in the order the kernel's loads visit them
      for (int mm = 0; mm * lpr < nch; ++mm)
        for (int h = 0; h < 4; ++h)
          for (int l = 0; l < lpr; ++l) {
            const int ch = l + lpr * mm;
            if (ch < nch) slot.push_back((unsigned)(4 * ch + h));
          }
      const size_t base = idx.size();
      idx.resize(base + rowv.size());
      for (size_t r = 0; r < rowv.size(); ++r) idx[base + slot[r]] = rowv[r];
      ptr4[i + 1] = (int)idx.size();
    }
    if (fits && idx.size() <= (size_t)INT32_MAX - 4096) {
      const unsigned zero = (unsigned)tab.size() << 16;                 // j = 0 with G = 0
      tab.push_back(make_float4(0.f, 0.f, 0.f, 0.f));
      for (unsigned& v : idx)
        if (v == kPad) v = zero;
      if (idx.empty()) idx.assign(4, zero);                             // never a null pointer
      CPM_TRY(upload(&c->ee_ptr, ptr4, st));
      CPM_TRY(upload(&c->ee_idx, idx, st));
      CPM_TRY(upload(&c->ee_tab, tab, st));
      c->ee_ntab = (int)tab.size();
      c->ee_lpr = lpr;
      return CPM_OK;
    }
  }
  CPM_TRY(upload(&c->ee_ptr, ptr, st));
  CPM_TRY(upload(&c->ee_g, ent, st));
  return CPM_OK;
}

static int build(cpm_ctx* c, int32_t ne, const double* xyz, const int32_t* side, const int32_t* cell,
                 cudaStream_t st, const void* image = nullptr, int64_t image_bytes = 0) {
  const cpm_params& p = c->p;
  c->ne = ne;
  c->ncons = (p.geometry == CPM_DOUBLED) ? 2 : 1;
  c->mixed = (p.precision == CPM_MIXED);
  for (int d = 0; d < 3; ++d) c->ebox[d] = p.box[d];
  if (p.geometry == CPM_SLAB) c->ebox[2] *= p.slab_factor;
  c->V = c->ebox[0] * c->ebox[1] * c->ebox[2];
  c->Lz = p.box[2];
  c->P = p.spme_order;
  for (int d = 0; d < 3; ++d) c->K[d] = p.grid[d];
  c->Mr = (long long)c->K[0] * c->K[1] * c->K[2];
  c->Mc = (long long)c->K[0] * c->K[1] * (c->K[2] / 2 + 1);
  c->Mr_s = (c->Mr + 63) & ~63LL;
  c->Mc_s = (c->Mc + 31) & ~31LL;
  CPM_CUDA(cudaGetDevice(&c->dev));

  // real-space cell grid: edge >= rcut/2, stencil half-width ceil(rcut/edge)
  c->ncell = 1;
  for (int d = 0; d < 3; ++d) {
    c->nc[d] = std::max(1, (int)std::floor(c->ebox[d] / (0.5 * p.rcut)));
    c->edge[d] = c->ebox[d] / c->nc[d];
    c->sten[d] = (int)std::ceil(p.rcut / c->edge[d] - 1e-12);
    c->ncell *= c->nc[d];
  }
  if ((2 * c->sten[0] + 1) * (2 * c->sten[1] + 1) * (2 * c->sten[2] + 1) > kMaxStencil) {
    set_error("the cell is too small for rcut: the neighbour stencil exceeds %d cells", kMaxStencil);
    return CPM_ERR_ARG;
  }

  // ---------------- electrode host data ----------------
  std::vector<double4_32a> pos(ne);
  std::vector<double> zraw(ne), v(ne), c1(ne, 0.0), eplus(ne, 0.0);
  for (int i = 0; i < ne; ++i) {
    pos[i] = make_double4_32a(wrap_coord(xyz[3 * i], c->ebox[0]), wrap_coord(xyz[3 * i + 1], c->ebox[1]),
                          wrap_coord(xyz[3 * i + 2], c->ebox[2]), 0.0);
    zraw[i] = xyz[3 * i + 2];
    const double d = 0.5 * side[i];
    v[i] = (p.geometry == CPM_FF) ? d - zraw[i] / c->Lz : d;
    if (p.geometry == CPM_DOUBLED) c1[i] = cell[i] == 1 ? 1.0 : 0.0;
    eplus[i] = side[i] > 0 ? 1.0 : 0.0;
  }
  // cell sort (stable by index)
  std::vector<int> flat(ne), count(c->ncell + 1, 0);
  std::vector<int4> cc(ne);
  for (int i = 0; i < ne; ++i) {
    int ci[3];
    const double r[3] = {pos[i].x, pos[i].y, pos[i].z};
    for (int d = 0; d < 3; ++d) ci[d] = std::min(c->nc[d] - 1, std::max(0, (int)std::floor(r[d] / c->edge[d])));
    flat[i] = (ci[0] * c->nc[1] + ci[1]) * c->nc[2] + ci[2];
    cc[i] = make_int4(ci[0], ci[1], ci[2], flat[i]);
    count[flat[i] + 1]++;
  }
  for (int k = 0; k < c->ncell; ++k) count[k + 1] += count[k];
  std::vector<int> start(count.begin(), count.end()), cursor(count.begin(), count.end() - 1);
  std::vector<int> sorted(ne);
  std::vector<double4_32a> loc64(ne);
  std::vector<float4> loc32(ne);
  std::vector<int4> cellc(ne);
  for (int i = 0; i < ne; ++i) {
    const int s = cursor[flat[i]]++;
    sorted[s] = i;
    const double lx = pos[i].x - cc[i].x * c->edge[0], ly = pos[i].y - cc[i].y * c->edge[1],
                 lz = pos[i].z - cc[i].z * c->edge[2];
    loc64[s] = make_double4_32a(lx, ly, lz, 0.0);
    loc32[s] = make_float4((float)lx, (float)ly, (float)lz, 0.0f);
    cellc[s] = cc[i];
  }
  // fixed B-spline stencils (original order)
  std::vector<int4> base(ne);
  std::vector<double> th((size_t)ne * 3 * PMAX), dth((size_t)ne * 3 * PMAX);
  std::vector<float> th32(th.size()), dth32(th.size());
  for (int i = 0; i < ne; ++i) {
    const double r[3] = {pos[i].x, pos[i].y, pos[i].z};
    int i0[3];
    for (int d = 0; d < 3; ++d) {
      const double u = r[d] / c->ebox[d] * c->K[d];
      const double fl = std::floor(u);
      i0[d] = (int)fl;
      double w[PMAX], dw[PMAX];
      bspline_host(u - fl, c->P, w, dw);
      for (int t = 0; t < PMAX; ++t) {
        const size_t o = ((size_t)i * 3 + d) * PMAX + t;
        th[o] = w[t];
        dth[o] = dw[t];
        th32[o] = (float)w[t];
        dth32[o] = (float)dw[t];
      }
    }
    base[i] = make_int4(i0[0], i0[1], i0[2], 0);
  }
  CPM_TRY(upload(&c->e_pos64, pos, st));
  CPM_TRY(upload(&c->e_loc64, loc64, st));
  CPM_TRY(upload(&c->e_loc32, loc32, st));
  CPM_TRY(upload(&c->e_cellc, cellc, st));
  CPM_TRY(upload(&c->e_sorted, sorted, st));
  CPM_TRY(upload(&c->e_start, start, st));
  CPM_TRY(upload(&c->e_base, base, st));
  CPM_TRY(upload(&c->e_th64, th, st));
  CPM_TRY(upload(&c->e_dth64, dth, st));
  CPM_TRY(upload(&c->e_th32, th32, st));
  CPM_TRY(upload(&c->e_dth32, dth32, st));
  CPM_TRY(upload(&c->e_z, zraw, st));
  CPM_TRY(upload(&c->e_v, v, st));
  CPM_TRY(upload(&c->e_c1, c1, st));
  CPM_TRY(upload(&c->e_plus, eplus, st));
  if (c->mixed) CPM_TRY(build_ee_list(c, pos, cc, start, sorted, st));

  // ---------------- SPME influence function (the mesh form of A uses it) ----------------
  {
    std::vector<double> G;
    influence_host(c, G);
    CPM_TRY(upload(&c->G64, G, st));
    std::vector<float> G32(G.begin(), G.end());
    CPM_TRY(upload(&c->G32, G32, st));
  }
  // ---------------- A, its inverse and the projection pieces (float64) ----------------
  CPM_LIB(cublasCreate(&c->cublas) == CUBLAS_STATUS_SUCCESS, "cublasCreate");
  CPM_LIB(cublasSetStream(c->cublas, st) == CUBLAS_STATUS_SUCCESS, "cublasSetStream");
  CPM_LIB(cusolverDnCreate(&c->solver) == CUSOLVER_STATUS_SUCCESS, "cusolverDnCreate");
  CPM_LIB(cusolverDnSetStream(c->solver, st) == CUSOLVER_STATUS_SUCCESS, "cusolverDnSetStream");
  c->ldb = (ne + 3) & ~3;
  c->mirror = false;
  if (p.geometry == CPM_DOUBLED && p.dc_blocks != CPM_DC_FULL) {
    c->mirror = find_mirror(c, pos, cell);
    if (!c->mirror && p.dc_blocks == CPM_DC_MIRROR) {
      set_error("dc_blocks = CPM_DC_MIRROR, but the sub-cell-1 electrode is not the z-mirror image of sub-cell 0");
      return CPM_ERR_ARG;
    }
    c->nh = ne / 2;
  }
  if (image) CPM_TRY(load_image(c, image, image_bytes, matrix_key(&p, ne, xyz, side, cell), st));
  else if (c->mirror) CPM_TRY(build_mirror(c, pos, v, side, st));
  else CPM_TRY(build_full(c, v, c1, side, st));

  // ---------------- SPME ----------------
  {
    // mesh coordinate of every cell origin, split into an integer and a fraction per axis, so the
    // per-step kernels only add the (small) cell-local offset in the working precision
    std::vector<int> sI;
    std::vector<double> sF;
    std::vector<float> sF32;
    for (int d = 0; d < 3; ++d)
      for (int cidx = 0; cidx < c->nc[d]; ++cidx) {
        const double u0 = (double)cidx * c->K[d] / c->nc[d];
        const double fl = std::floor(u0);
        sI.push_back((int)fl);
        sF.push_back(u0 - fl);
        sF32.push_back((float)(u0 - fl));
      }
    CPM_TRY(upload(&c->spl_I, sI, st));
    CPM_TRY(upload(&c->spl_F64, sF, st));
    CPM_TRY(upload(&c->spl_F32, sF32, st));
  }
  CPM_TRY(make_plans(c));
  CPM_TRY(cpm_internal_alloc_step_buffers(c));
  CPM_CUDA(cudaStreamSynchronize(st));
  return CPM_OK;
}

}  // namespace cpm

// ------------------------------------------------------------------------------------------
// C ABI
// ------------------------------------------------------------------------------------------
extern "C" int cpm_build_matrix(const cpm_params* p, int32_t n_elec, const double* elec_xyz_host,
                                const int32_t* elec_side_host, const int32_t* elec_cell_host, void* stream,
                                cpm_ctx** out) {
  if (!out) return CPM_ERR_ARG;
  *out = nullptr;
  const int v = cpm::validate(p, n_elec, elec_xyz_host, elec_side_host, elec_cell_host);
  if (v != CPM_OK) {
    cpm::set_error("cpm_build_matrix: invalid parameters or electrode input");
    return v;
  }
  cpm_ctx* c = new (std::nothrow) cpm_ctx();
  if (!c) return CPM_ERR_NOMEM;
  c->p = *p;
  c->key = cpm::matrix_key(p, n_elec, elec_xyz_host, elec_side_host, elec_cell_host);
  const int s = cpm::build(c, n_elec, elec_xyz_host, elec_side_host, elec_cell_host, (cudaStream_t)stream);
  if (s != CPM_OK) {
    cudaStreamSynchronize((cudaStream_t)stream);
    cpm_destroy(c);
    return s;
  }
  *out = c;
  return CPM_OK;
}

extern "C" int cpm_matrix_key(const cpm_params* p, int32_t n_elec, const double* elec_xyz_host,
                              const int32_t* elec_side_host, const int32_t* elec_cell_host, uint64_t* key) {
  if (!key) return CPM_ERR_ARG;
  const int v = cpm::validate(p, n_elec, elec_xyz_host, elec_side_host, elec_cell_host);
  if (v != CPM_OK) {
    cpm::set_error("cpm_matrix_key: invalid parameters or electrode input");
    return v;
  }
  *key = cpm::matrix_key(p, n_elec, elec_xyz_host, elec_side_host, elec_cell_host);
  return CPM_OK;
}

extern "C" int cpm_matrix_image(const cpm_ctx* c, void* host_out, int64_t* bytes) {
  if (!c || !bytes) {
    cpm::set_error("cpm_matrix_image: null argument");
    return CPM_ERR_ARG;
  }
  const int rows = c->mirror ? 2 * c->nh : c->ne;
  const int64_t nS = (int64_t)rows * c->ld64, nW = c->mirror ? 4LL * c->nh : 2LL * c->ne, nSv = rows;
  const int64_t need = (int64_t)sizeof(cpm::ImageHeader) + 8 * (nS + nW + nSv);
  if (!host_out) {
    *bytes = need;
    return CPM_OK;
  }
  if (*bytes < need) {
    cpm::set_error("cpm_matrix_image: buffer of %lld bytes, %lld needed", (long long)*bytes, (long long)need);
    return CPM_ERR_ARG;
  }
  cpm::ImageHeader h;
  std::memset(&h, 0, sizeof h);
  std::memcpy(h.magic, cpm::kImageMagic, 8);
  h.key = c->key;
  h.ne = c->ne;
  h.ncons = c->ncons;
  h.mirror = c->mirror ? 1 : 0;
  h.nh = c->nh;
  h.ld64 = c->ld64;
  h.nS = nS;
  h.nW = nW;
  h.nSv = nSv;
  for (int k = 0; k < 4; ++k) h.Mh[k] = c->Mh[k];
  h.WTv[0] = c->WTv[0];
  h.WTv[1] = c->WTv[1];
  h.dqdpsi = c->dqdpsi;
  char* dst = static_cast<char*>(host_out);
  std::memcpy(dst, &h, sizeof h);
  double* body = reinterpret_cast<double*>(dst + sizeof h);
  CPM_CUDA(cudaMemcpy(body, c->S64, sizeof(double) * nS, cudaMemcpyDeviceToHost));
  CPM_CUDA(cudaMemcpy(body + nS, c->W, sizeof(double) * nW, cudaMemcpyDeviceToHost));
  CPM_CUDA(cudaMemcpy(body + nS + nW, c->Sv, sizeof(double) * nSv, cudaMemcpyDeviceToHost));
  *bytes = need;
  return CPM_OK;
}

extern "C" int cpm_build_matrix_from_image(const cpm_params* p, int32_t n_elec, const double* elec_xyz_host,
                                           const int32_t* elec_side_host, const int32_t* elec_cell_host,
                                           const void* image_host, int64_t image_bytes, void* stream,
                                           cpm_ctx** out) {
  if (!out) return CPM_ERR_ARG;
  *out = nullptr;
  if (!image_host) {
    cpm::set_error("cpm_build_matrix_from_image: null image");
    return CPM_ERR_ARG;
  }
  const int v = cpm::validate(p, n_elec, elec_xyz_host, elec_side_host, elec_cell_host);
  if (v != CPM_OK) {
    cpm::set_error("cpm_build_matrix_from_image: invalid parameters or electrode input");
    return v;
  }
  cpm_ctx* c = new (std::nothrow) cpm_ctx();
  if (!c) return CPM_ERR_NOMEM;
  c->p = *p;
  c->key = cpm::matrix_key(p, n_elec, elec_xyz_host, elec_side_host, elec_cell_host);
  const int s = cpm::build(c, n_elec, elec_xyz_host, elec_side_host, elec_cell_host, (cudaStream_t)stream,
                           image_host, image_bytes);
  if (s != CPM_OK) {
    cudaStreamSynchronize((cudaStream_t)stream);
    cpm_destroy(c);
    return s;
  }
  *out = c;
  return CPM_OK;
}

extern "C" void cpm_destroy(cpm_ctx* c) {
  if (!c) return;
  cpm_profile_enable(c, 0);
  void* bufs[] = {c->e_pos64, c->e_loc64, c->e_loc32, c->e_cellc, c->e_sorted, c->e_start, c->e_base,
                  c->e_th64, c->e_dth64, c->e_th32, c->e_dth32, c->e_z, c->e_v, c->e_c1, c->e_plus, c->S64, c->S32,
                  c->W, c->Sv, c->G64, c->G32, c->mesh_r, c->mesh_c, c->mesh_phi, c->l_cell, c->l_count,
                  c->l_start, c->l_sorted, c->l_loc64, c->l_loc32, c->l_tmp, c->qT, c->spl_I,
                  c->spl_F64, c->spl_F32, c->phi_real, c->b_tmp, c->b32, c->qraw32, c->f_pair,
                  c->scal, c->status, c->m_i0, c->m_j, c->e_c1m, c->ypm, c->qpm, c->qpart, c->fft_tw, c->br_pad, c->sym_S, c->ee_ptr, c->ee_g,
                  c->ee_idx, c->ee_tab, c->e_field, c->f_sorted32, c->sym_w32, c->sym_c1f};
  for (void* b : bufs)
    if (b) cudaFree(b);
  for (int b = 0; b < 2; ++b)
    if (c->have_plan[b]) {
      cufftDestroy(c->plan_r2c[b]);
      cufftDestroy(c->plan_c2r[b]);
    }
  if (c->ev_fork) cudaEventDestroy(c->ev_fork);
  if (c->ev_join) cudaEventDestroy(c->ev_join);
  if (c->ev_sorted) cudaEventDestroy(c->ev_sorted);
  if (c->ev_ee) cudaEventDestroy(c->ev_ee);
  if (c->side) cudaStreamDestroy(c->side);
  if (c->cublas) cublasDestroy(c->cublas);
  if (c->solver) cusolverDnDestroy(c->solver);
  delete c;
}

extern "C" int cpm_capacitance(const cpm_ctx* c, double* out) {
  if (!c || !out) return CPM_ERR_ARG;
  *out = c->dqdpsi;
  return CPM_OK;
}

extern "C" int cpm_copy_matrix(const cpm_ctx* c, int32_t which, double* host_out) {
  if (!c || !host_out) return CPM_ERR_ARG;
  if (c->mirror) {
    // q_I0 = (q+ + q-) / 2, q_J = (q+ - q-) / 2 with q+- = S+- (y_I0 +- y_J): S(I0, I0) = S(J, J) =
    // (S+ + S-) / 2, S(I0, J) = S(J, I0) = (S+ - S-) / 2; A^-1 e = (w+, w+), A^-1 e_1 = ((w+ - w-)/2, (w+ + w-)/2)
    const int N = c->nh, ne = c->ne;
    const std::vector<int>& I = c->h_i0;
    const std::vector<int>& J = c->h_j;
    if (which == 0) {
      std::vector<double> S((size_t)2 * N * c->ldh);
      CPM_CUDA(cudaMemcpy(S.data(), c->S64, sizeof(double) * S.size(), cudaMemcpyDeviceToHost));
      const double* Sp = S.data();
      const double* Sm = S.data() + (size_t)N * c->ldh;
      for (int k = 0; k < N; ++k)
        for (int l = 0; l < N; ++l) {
          const double sp = Sp[(size_t)k * c->ldh + l], sm = Sm[(size_t)k * c->ldh + l];
          host_out[(size_t)I[k] * ne + I[l]] = 0.5 * (sp + sm);
          host_out[(size_t)J[k] * ne + J[l]] = 0.5 * (sp + sm);
          host_out[(size_t)I[k] * ne + J[l]] = 0.5 * (sp - sm);
          host_out[(size_t)J[k] * ne + I[l]] = 0.5 * (sp - sm);
        }
    } else if (which == 1) {
      std::vector<double> sv(2 * (size_t)N);
      CPM_CUDA(cudaMemcpy(sv.data(), c->Sv, sizeof(double) * sv.size(), cudaMemcpyDeviceToHost));
      for (int k = 0; k < N; ++k) {
        host_out[I[k]] = 0.5 * (sv[k] + sv[N + k]);
        host_out[J[k]] = 0.5 * (sv[k] - sv[N + k]);
      }
    } else if (which == 2) {
      std::vector<double> w(4 * (size_t)N);
      CPM_CUDA(cudaMemcpy(w.data(), c->W, sizeof(double) * w.size(), cudaMemcpyDeviceToHost));
      for (int k = 0; k < N; ++k) {
        const double wp = w[2 * k], wm = w[2 * (size_t)N + 2 * k + 1];
        host_out[(size_t)I[k] * 2 + 0] = wp;
        host_out[(size_t)J[k] * 2 + 0] = wp;
        host_out[(size_t)I[k] * 2 + 1] = 0.5 * (wp - wm);
        host_out[(size_t)J[k] * 2 + 1] = 0.5 * (wp + wm);
      }
    } else {
      return CPM_ERR_ARG;
    }
    return CPM_OK;
  }
  if (which == 0) {
    CPM_CUDA(cudaMemcpy2D(host_out, sizeof(double) * c->ne, c->S64, sizeof(double) * c->ld64,
                          sizeof(double) * c->ne, c->ne, cudaMemcpyDeviceToHost));
  } else if (which == 1) {
    CPM_CUDA(cudaMemcpy(host_out, c->Sv, sizeof(double) * c->ne, cudaMemcpyDeviceToHost));
  } else if (which == 2) {
    std::vector<double> w((size_t)c->ne * 2);
    CPM_CUDA(cudaMemcpy(w.data(), c->W, sizeof(double) * c->ne * 2, cudaMemcpyDeviceToHost));
    for (int i = 0; i < c->ne; ++i)
      for (int k = 0; k < c->ncons; ++k) host_out[(size_t)i * c->ncons + k] = w[2 * i + k];
  } else {
    return CPM_ERR_ARG;
  }
  return CPM_OK;
}

extern "C" int cpm_matrix_layout(const cpm_ctx* c, int32_t* mirror_blocks, int64_t* s_bytes) {
  if (!c) return CPM_ERR_ARG;
  if (mirror_blocks) *mirror_blocks = c->mirror ? 1 : 0;
  if (s_bytes) {
    if (c->sym_ok && (c->sapply_variant == CPM_SAPPLY_SYM || c->sapply_variant == CPM_SAPPLY_SYM_TMA)) {
      const long long nt = c->sym_nt;
      *s_bytes = (c->mirror ? 2LL : 1LL) * (nt * (nt + 1) / 2) * 128LL * 128LL * 4LL;
    } else {
      const long long rows = c->mirror ? 2LL * c->nh : (long long)c->ne;
      *s_bytes = rows * (long long)c->ld64 * (c->mixed ? 4 : 8);
    }
  }
  return CPM_OK;
}

extern "C" int cpm_pair_list_layout(const cpm_ctx* c, int64_t* pairs, int32_t* table) {
  if (!c) return CPM_ERR_ARG;
  const bool any = c->ee_g != nullptr || c->ee_idx != nullptr;
  if (pairs) *pairs = any ? c->ee_nnz : 0;
  if (table) *table = c->ee_idx ? c->ee_ntab : 0;
  return CPM_OK;
}

extern "C" int cpm_info(const cpm_ctx* c, int32_t* n_elec, int32_t* ncons, int64_t* mesh_points,
                        int32_t* n_cells) {
  if (!c) return CPM_ERR_ARG;
  if (n_elec) *n_elec = c->ne;
  if (ncons) *ncons = c->ncons;
  if (mesh_points) *mesh_points = c->Mr;
  if (n_cells) *n_cells = c->ncell;
  return CPM_OK;
}

extern "C" int cpm_status(cpm_ctx* c, void* stream) {
  if (!c) return CPM_ERR_ARG;
  int h = 0;
  CPM_CUDA(cudaStreamSynchronize((cudaStream_t)stream));
  CPM_CUDA(cudaMemcpy(&h, c->status, sizeof(int), cudaMemcpyDeviceToHost));
  CPM_CUDA(cudaMemset(c->status, 0, sizeof(int)));
  if (h & cpm::DE_NONFINITE) return CPM_ERR_NONFINITE;
  if (h & cpm::DE_DOMAIN) return CPM_ERR_DOMAIN;
  if (h & cpm::DE_CAPACITY) return CPM_ERR_CAPACITY;
  if (h & cpm::DE_TIMEOUT) return CPM_ERR_TIMEOUT;
  return CPM_OK;
}

extern "C" const char* cpm_strerror(int s) {
  switch (s) {
    case CPM_OK: return "ok";
    case CPM_ERR_ARG: return "invalid argument";
    case CPM_ERR_CUDA: return "CUDA runtime error";
    case CPM_ERR_NOT_SPD: return "elastance matrix is not positive definite";
    case CPM_ERR_NONFINITE: return "non-finite coordinate or charge";
    case CPM_ERR_CAPACITY: return "replica count or site count above build-time capacity";
    case CPM_ERR_DOMAIN: return "electrolyte site outside [0, L_z) in z";
    case CPM_ERR_TIMEOUT: return "bounded device wait timed out";
    case CPM_ERR_LIBRARY: return "cuFFT / cuBLAS / cuSOLVER error";
    case CPM_ERR_NOMEM: return "out of device memory";
    default: return "unknown status";
  }
}

extern "C" const char* cpm_last_error(void) { return cpm::g_last_error.c_str(); }
