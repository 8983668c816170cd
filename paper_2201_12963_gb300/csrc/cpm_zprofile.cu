// Laterally averaged charge density rho(z) and potential psi(z) across the cell (Sec. II.C).
//
// rho: nbins bins of width h = L_z / nbins over the Ewald box in z (x, y averaged), float64.
//   Electrolyte point charges go to the bin of their wrapped z; an electrode site's Gaussian charge
//   (Eq. 2) is integrated over every bin within 6.5 / eta of its centre (z-projection
//   q eta / sqrt(pi) exp(-eta^2 (z - z_i)^2), differences of erf; the part beyond is below 4e-20 q),
//   periodic images by wrapping the bin index.  Densities per bin volume L_x L_y h; the call adds
//   into rho, so repeated calls accumulate a time average (pass 1 / samples to cpm_potential_z).
// psi: the 1-D Poisson equation psi'' = -4 pi k_e rho on the bin centres with the periodic second
//   difference.  With g_i = psi_{i+1} - psi_i the difference equations read g_i - g_{i-1} = h^2 f_i,
//   f = -4 pi k_e rho (mean removed: the cell is neutral), so g is a prefix sum of h^2 f plus the
//   constant that makes sum_i g_i = 0 (periodicity), and psi is a prefix sum of g, shifted to zero
//   mean: the same solution as inverting the finite-difference matrix.  Finite field: plus the ramp
//   dpsi (i + 1/2) h / L_z (a jump of dpsi across the cell boundary); doubled cell, slab: continuity.
#include "cpm_internal.cuh"

#include <algorithm>

namespace cpm {

constexpr int PZ_THREADS = 1024;

__global__ void __launch_bounds__(256) k_rho_elyt(const int* __restrict__ off, const double* __restrict__ xyzq,
                                                  int cap, double box_z, double inv_box_z, int nbins, double w,
                                                  double* __restrict__ rho) {
  const int rep = blockIdx.y;
  const int o = off[rep];
  const int n = min(off[rep + 1] - o, cap);
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const double4_32a s = reinterpret_cast<const double4_32a*>(xyzq)[o + i];
  if (!(isfinite(s.z) && isfinite(s.w))) return;
  const double z = s.z - box_z * floor(s.z * inv_box_z);
  const int b = min(nbins - 1, max(0, (int)(z * nbins * inv_box_z)));
  atomicAdd(&rho[(size_t)rep * nbins + b], s.w * w);
}

// One warp per electrode site: the bins within reach of its Gaussian.
__global__ void __launch_bounds__(256) k_rho_elec(const double* __restrict__ ez, const double* __restrict__ q, int ne,
                                                  double box_z, int nbins, double eta, int reach, double w,
                                                  double* __restrict__ rho) {
  const int rep = blockIdx.y;
  const int lane = threadIdx.x & 31;
  const double h = box_z / nbins;
  for (int i = (blockIdx.x * blockDim.x + threadIdx.x) >> 5; i < ne; i += (gridDim.x * blockDim.x) >> 5) {
    const double c = ez[i] - box_z * floor(ez[i] / box_z);
    const double qi = q[(size_t)rep * ne + i];
    const int u0 = (int)floor(c / h);
    for (int k = lane; k <= 2 * reach; k += 32) {
      const int u = u0 - reach + k;                  // unwrapped bin
      const double lo = u * h, hi = lo + h;
      const double frac = 0.5 * (erf(eta * (hi - c)) - erf(eta * (lo - c)));
      const int b = ((u % nbins) + nbins) % nbins;
      atomicAdd(&rho[(size_t)rep * nbins + b], qi * frac * w);
    }
  }
}

// Block-wide inclusive prefix sum of x[0..n) in place (float64), chunked per thread.
__device__ void block_scan(double* x, int n, double* part) {
  const int t = threadIdx.x, nt = blockDim.x;
  const int chunk = (n + nt - 1) / nt;
  const int b = t * chunk, e = min(n, b + chunk);
  double s = 0.0;
  for (int k = b; k < e; ++k) s += x[k];
  part[t] = s;
  __syncthreads();
  for (int o = 1; o < nt; o <<= 1) {
    const double v = t >= o ? part[t - o] : 0.0;
    __syncthreads();
    part[t] += v;
    __syncthreads();
  }
  double run = part[t] - s;
  for (int k = b; k < e; ++k) {
    run += x[k];
    x[k] = run;
  }
  __syncthreads();
}

__device__ double block_mean(const double* x, int n, double* part) {
  double s = 0.0;
  for (int k = threadIdx.x; k < n; k += blockDim.x) s += x[k];
  part[threadIdx.x] = s;
  __syncthreads();
  for (int o = blockDim.x / 2; o > 0; o >>= 1) {
    if (threadIdx.x < o) part[threadIdx.x] += part[threadIdx.x + o];
    __syncthreads();
  }
  const double m = part[0] / n;
  __syncthreads();
  return m;
}

// One block per replica; work arrays in dynamic shared memory (nbins float64).
__global__ void __launch_bounds__(PZ_THREADS) k_poisson_z(const double* __restrict__ rho, int nbins, double scale,
                                                          double box_z, const double* __restrict__ dpsi, int ramp,
                                                          double* __restrict__ psi) {
  extern __shared__ double pz[];                    // [nbins]
  __shared__ double part[PZ_THREADS];
  const int rep = blockIdx.x;
  const double h = box_z / nbins;
  const double* r = rho + (size_t)rep * nbins;
  for (int k = threadIdx.x; k < nbins; k += blockDim.x) pz[k] = -4.0 * PI * KE * r[k] * scale * h * h;
  __syncthreads();
  const double mf = block_mean(pz, nbins, part);
  for (int k = threadIdx.x; k < nbins; k += blockDim.x) pz[k] -= mf;
  __syncthreads();
  block_scan(pz, nbins, part);                      // s_i
  const double ms = block_mean(pz, nbins, part);
  for (int k = threadIdx.x; k < nbins; k += blockDim.x) pz[k] -= ms;     // g_i = s_i - mean(s)
  __syncthreads();
  block_scan(pz, nbins, part);                      // inclusive: psi_{i+1} - psi_0
  // psi_0 = 0, psi_i = (inclusive sum up to i - 1); shift to zero mean
  double* out = psi + (size_t)rep * nbins;
  for (int k = threadIdx.x; k < nbins; k += blockDim.x) out[k] = k == 0 ? 0.0 : pz[k - 1];
  __syncthreads();
  double s = 0.0;
  for (int k = threadIdx.x; k < nbins; k += blockDim.x) s += out[k];
  part[threadIdx.x] = s;
  __syncthreads();
  for (int o = blockDim.x / 2; o > 0; o >>= 1) {
    if (threadIdx.x < o) part[threadIdx.x] += part[threadIdx.x + o];
    __syncthreads();
  }
  const double mp = part[0] / nbins;
  const double slope = ramp ? dpsi[rep] / box_z : 0.0;
  for (int k = threadIdx.x; k < nbins; k += blockDim.x) out[k] = out[k] - mp + slope * (k + 0.5) * h;
}

}  // namespace cpm

using namespace cpm;

extern "C" int cpm_density_z(cpm_ctx* c, int32_t n_rep, const int32_t* off, const double* xyzq, const double* q,
                             int32_t nbins, double* rho, void* stream) {
  if (!c || !off || !xyzq || !q || !rho || n_rep < 1 || n_rep > c->p.max_replicas || nbins < 4) {
    set_error("cpm_density_z: null pointer or size out of range");
    return CPM_ERR_ARG;
  }
  cudaStream_t st = (cudaStream_t)stream;
  const double bz = c->ebox[2];
  const double w = 1.0 / (c->ebox[0] * c->ebox[1] * (bz / nbins));
  const int cap = c->p.max_elyt;
  k_rho_elyt<<<dim3((cap + 255) / 256, n_rep), 256, 0, st>>>(off, xyzq, cap, bz, 1.0 / bz, nbins, w, rho);
  CPM_LAUNCH();
  const int reach = (int)std::ceil(6.5 / c->p.eta / (bz / nbins)) + 1;
  const int blocks = std::min(152 * 8, (c->ne * 32 + 255) / 256);
  k_rho_elec<<<dim3(blocks, n_rep), 256, 0, st>>>(c->e_z, q, c->ne, bz, nbins, c->p.eta, reach, w, rho);
  CPM_LAUNCH();
  return CPM_OK;
}

extern "C" int cpm_potential_z(cpm_ctx* c, int32_t n_rep, int32_t nbins, const double* rho, double scale,
                               const double* dpsi, double* psi, void* stream) {
  if (!c || !rho || !dpsi || !psi || n_rep < 1 || nbins < 4 || (size_t)nbins * sizeof(double) > 96 * 1024) {
    set_error("cpm_potential_z: null pointer or size out of range (nbins <= 12288)");
    return CPM_ERR_ARG;
  }
  const size_t smem = sizeof(double) * (size_t)nbins;
  if (smem > 48 * 1024)
    CPM_CUDA(cudaFuncSetAttribute(k_poisson_z, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
  k_poisson_z<<<n_rep, PZ_THREADS, smem, (cudaStream_t)stream>>>(rho, nbins, scale, c->ebox[2], dpsi,
                                                                 c->p.geometry == CPM_FF ? 1 : 0, psi);
  CPM_LAUNCH();
  return CPM_OK;
}
