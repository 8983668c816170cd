// Molecular dynamics around the CPM step (Appendix A: velocity-Verlet at 2 fs with a Nose-Hoover
// thermostat on the electrolyte, one per sub-cell of the doubled cell; Appendix B: electrode charges
// re-solved every 5 steps and held in between).  The electrode is frozen; each electrolyte site is
// a point ion with a Lennard-Jones type.
//
// Integrator (per step, all on the caller's stream):
//   thermostat half step(s) -> combined velocity scale s per (replica, group)      k_md_kick_ke (last block)
//   v = s v + dt/2 F/m ; x += dt v ; x, y wrapped into the cell                    k_md_kick_drift
//   forces at the new positions: cpm_step (charges re-solved when the step index is a multiple of
//     k) or cpm_forces (charges held), the Lennard-Jones term added by the same force pass
//   v += dt/2 F/m and the kinetic energy per (replica, group), then the thermostat   k_md_kick_ke
// The thermostat is one Nose-Hoover variable per group, propagated by the symmetric Trotter
// splitting of Martyna, Tuckerman, Tobias and Klein (Mol. Phys. 87, 1117 (1996)): a half step is a
// quarter-step update of v_xi, the scaling exp(-v_xi dt / 2), xi += v_xi dt / 2 and a second
// quarter step; Q = g k_B T tau^2 with g = 3 N_group.  The trailing half step of one time step and
// the leading half step of the next are taken together, so their velocity scales multiply into the
// next kick; the last trailing scale of a call is applied by k_md_scale.
//
// Lennard-Jones: Lorentz-Berthelot mixing, force-shifted at the cutoff (energy and force continuous),
// electrolyte-electrolyte and electrolyte-electrode pairs, summed over every periodic image within
// the cutoff (<= the real-space Coulomb cutoff).  The run hands the parameters to the context for
// its duration; the step's real-space pair kernel for electrolyte targets evaluates them on the
// same staged sources as the Coulomb pairs (k_pair_cell with LJ), so the force gather of the step
// returns the sum.
#include "cpm_internal.cuh"

#include <algorithm>
#include <cmath>
#include <vector>

namespace cpm {

constexpr double KB_EV = 8.617333262e-5;             // Boltzmann constant, eV / K
constexpr double MVV2E = 103.64269652680505;         // 1 amu A^2 / fs^2 in eV
constexpr int kMdMaxGroups = 4;

// ------------------------------------------------------------------------------------------
// integrator kernels (float64)
// ------------------------------------------------------------------------------------------
// Per-type table in device memory: [0, kLjMaxTypes) dt / 2 / (m MVV2E), the velocity change per
// unit force in half a step; [kLjMaxTypes, 2 kLjMaxTypes) m MVV2E / 2, the kinetic energy per v^2.
constexpr int MD_HALF_M = kLjMaxTypes;

__global__ void __launch_bounds__(256) k_md_kick_drift(int n, double* __restrict__ xyzq, double* __restrict__ vel,
                                                       const double* __restrict__ F, const int* __restrict__ type,
                                                       const int* __restrict__ slot, const double* __restrict__ s,
                                                       const double* __restrict__ mt, double dt, double bx, double by) {
  pdl_enter();
  const int j = blockIdx.x * blockDim.x + threadIdx.x;
  if (j >= n) return;
  const double h = mt[type[j]];
  const double sc = s ? s[slot[j]] : 1.0;
  double* v = vel + 3 * (size_t)j;
  double* x = xyzq + 4 * (size_t)j;
  const double v0 = fma(sc, v[0], h * F[3 * (size_t)j + 0]);
  const double v1 = fma(sc, v[1], h * F[3 * (size_t)j + 1]);
  const double v2 = fma(sc, v[2], h * F[3 * (size_t)j + 2]);
  v[0] = v0;
  v[1] = v1;
  v[2] = v2;
  double x0 = fma(dt, v0, x[0]), x1 = fma(dt, v1, x[1]);
  x0 -= bx * floor(x0 / bx);
  x1 -= by * floor(x1 / by);
  x[0] = x0 < bx ? x0 : 0.0;
  x[1] = x1 < by ? x1 : 0.0;
  x[2] = fma(dt, v2, x[2]);
}

constexpr int NH_LEAD = 1, NH_TRAIL = 2;

// Thermostat half step(s) of slot i on its kinetic energy K: the trailing half of one time step
// (NH_TRAIL) and / or the leading half of the next (NH_LEAD); writes the combined velocity scale
// and the kinetic energy after it.
__device__ __forceinline__ void nh_update(int i, int mode, double K, double* __restrict__ thermo,
                                          const double* __restrict__ ndof, const double* __restrict__ Qm, double kT,
                                          double dt, double* __restrict__ s_out, double* __restrict__ kcur) {
  double xi = thermo[2 * i], vxi = thermo[2 * i + 1];
  double stot = 1.0;
  const double g = ndof[i], Q = Qm[i];
  if (g > 0.0 && Q > 0.0) {
    for (int half = 0; half < 2; ++half) {
      if (!(mode & (half == 0 ? NH_TRAIL : NH_LEAD))) continue;
      vxi += 0.25 * dt * (2.0 * K - g * kT) / Q;
      const double s = exp(-0.5 * dt * vxi);
      K *= s * s;
      xi += 0.5 * dt * vxi;
      vxi += 0.25 * dt * (2.0 * K - g * kT) / Q;
      stot *= s;
    }
  }
  thermo[2 * i] = xi;
  thermo[2 * i + 1] = vxi;
  s_out[i] = stot;
  kcur[i] = K;
}

struct MdThermo {              // the thermostat step fused into k_md_kick_ke (mode 0: none)
  int mode, nslots;
  double* thermo;
  const double* ndof;
  const double* Qm;
  double kT, dt;
  double* s_out;
  double* kcur;
  unsigned int* done;          // blocks finished (the last one runs the thermostat and resets it)
};

// v += dt/2 F/m (kick != 0) and the kinetic energy per (replica, group) slot into ke (zero on
// entry).  With a thermostat step (th.mode != 0) the last block to finish applies it to every slot
// and zeroes ke for the next accumulation.
__global__ void __launch_bounds__(256) k_md_kick_ke(int n, double* __restrict__ vel, const double* __restrict__ F,
                                                    const int* __restrict__ type, const int* __restrict__ slot,
                                                    const double* __restrict__ mt, int kick, double* __restrict__ ke,
                                                    MdThermo th) {
  pdl_enter();
  const int j = blockIdx.x * blockDim.x + threadIdx.x;
  const int lane = threadIdx.x & 31;
  const bool valid = j < n;
  double e = 0.0;
  int sl = -1;
  if (valid) {
    const int ty = type[j];
    double* v = vel + 3 * (size_t)j;
    double v0 = v[0], v1 = v[1], v2 = v[2];
    if (kick) {
      const double h = mt[ty];
      v0 = fma(h, F[3 * (size_t)j + 0], v0);
      v1 = fma(h, F[3 * (size_t)j + 1], v1);
      v2 = fma(h, F[3 * (size_t)j + 2], v2);
      v[0] = v0;
      v[1] = v1;
      v[2] = v2;
    }
    e = mt[MD_HALF_M + ty] * (v0 * v0 + v1 * v1 + v2 * v2);
    sl = slot[j];
  }
  // segmented warp reduction over the (few) distinct slots of this warp
  unsigned todo = __ballot_sync(0xffffffffu, valid);
  while (todo) {
    const int leader = __ffs(todo) - 1;
    const int s = __shfl_sync(0xffffffffu, sl, leader);
    const bool mine = valid && sl == s;
    const double part = warp_sum(mine ? e : 0.0);
    if (lane == leader) atomicAdd(&ke[s], part);
    todo &= ~__ballot_sync(0xffffffffu, mine);
  }
  if (th.mode == 0) return;                       // uniform over the grid
  __shared__ bool last;
  __threadfence();                                // this block's sums are visible before its ticket
  __syncthreads();
  if (threadIdx.x == 0) last = atomicAdd(th.done, 1u) == gridDim.x - 1;
  __syncthreads();
  if (!last) return;
  __threadfence();
  for (int i = threadIdx.x; i < th.nslots; i += blockDim.x) {
    const double K = __ldcg(ke + i);
    nh_update(i, th.mode, K, th.thermo, th.ndof, th.Qm, th.kT, th.dt, th.s_out, th.kcur);
    ke[i] = 0.0;
  }
  if (threadIdx.x == 0) *th.done = 0u;
}

__global__ void __launch_bounds__(256) k_md_scale(int n, double* __restrict__ vel, const int* __restrict__ slot,
                                                  const double* __restrict__ s) {
  pdl_enter();
  const int j = blockIdx.x * blockDim.x + threadIdx.x;
  if (j >= n) return;
  const double sc = s[slot[j]];
  double* v = vel + 3 * (size_t)j;
  v[0] *= sc;
  v[1] *= sc;
  v[2] *= sc;
}

// Per replica: U, H, U_LJ, KE, thermostat energy, conserved total, temperature, Q_+.
__global__ void k_md_energy(int nrep, int ngroups, const double* __restrict__ e_coul, const double* __restrict__ scal,
                            const double* __restrict__ K, const double* __restrict__ thermo,
                            const double* __restrict__ ndof, const double* __restrict__ Qm, double kT, int thermostat,
                            double* __restrict__ out) {
  pdl_enter();
  const int rep = blockIdx.x * blockDim.x + threadIdx.x;
  if (rep >= nrep) return;
  double ke = 0.0, enh = 0.0, g = 0.0;
  for (int k = 0; k < ngroups; ++k) {
    const int i = rep * ngroups + k;
    ke += K[i];
    g += ndof[i];
    if (thermostat && Qm[i] > 0.0) enh += 0.5 * Qm[i] * thermo[2 * i + 1] * thermo[2 * i + 1] + ndof[i] * kT * thermo[2 * i];
  }
  const double U = e_coul[NENERGY * rep + 0], H = e_coul[NENERGY * rep + 1];
  const double ulj = scal[rep * NSCAL + S_E_LJ];
  double* o = out + CPM_MD_NENERGY * rep;
  o[0] = U;
  o[1] = H;
  o[2] = ulj;
  o[3] = ke;
  o[4] = enh;
  o[5] = ke + H + ulj + enh;
  o[6] = g > 0.0 ? 2.0 * ke / (g * KB_EV) : 0.0;
  o[7] = e_coul[NENERGY * rep + 3];
}

}  // namespace cpm

using namespace cpm;

#define MD_LAUNCH(ctx) \
  do {                 \
    ++(ctx)->launches; \
    CPM_LAUNCH();      \
  } while (0)

struct cpm_md {
  cpm_ctx* ctx = nullptr;
  cpm_md_params p;
  int nrep = 0, n = 0, ngroups = 1, nslots = 0;
  int* off = nullptr;          // [nrep + 1]
  int* type = nullptr;         // [n]
  int* slot = nullptr;         // [n] rep * ngroups + group
  double* F = nullptr;         // [n][3] forces at the current positions
  double* e_coul = nullptr;    // [nrep][NENERGY]
  double* thermo = nullptr;    // [nslots][2] (xi, v_xi)
  double* ke = nullptr;        // [nslots + 1]: kinetic energies, then the block counter of the fused thermostat
  double* kcur = nullptr;      // [nslots]
  double* s = nullptr;         // [nslots]
  double* ndof = nullptr;      // [nslots]
  double* Qm = nullptr;        // [nslots]
  double* mt = nullptr;        // [2 * kLjMaxTypes] per-type table (MD_HALF_M)
  LjSetup lj;
  long long step = 0;
  bool forces_valid = false;
};

static void md_free(cpm_md* m) {
  if (!m) return;
  void* ptrs[] = {m->off, m->type, m->slot, m->F, m->e_coul, m->thermo, m->ke, m->kcur, m->s, m->ndof, m->Qm, m->mt};
  for (void* p : ptrs)
    if (p) cudaFree(p);
  delete m;
}

static int md_check_params(const cpm_ctx* c, const cpm_md_params* p) {
  if (!(p->dt > 0.0 && std::isfinite(p->dt)) || p->charge_every < 1 || p->n_types < 1 ||
      p->n_types > CPM_MD_MAX_TYPES || p->n_groups < 1 || p->n_groups > kMdMaxGroups) {
    set_error("cpm_md_create: dt > 0, charge_every >= 1, 1 <= n_types <= %d, 1 <= n_groups <= %d required",
              CPM_MD_MAX_TYPES, kMdMaxGroups);
    return CPM_ERR_ARG;
  }
  for (int t = 0; t < p->n_types; ++t) {
    if (!(p->lj_sigma[t] >= 0.0 && std::isfinite(p->lj_sigma[t]) && p->lj_epsilon[t] >= 0.0 &&
          std::isfinite(p->lj_epsilon[t]) && std::isfinite(p->mass[t]))) {
      set_error("cpm_md_create: type %d: sigma, epsilon must be finite and >= 0", t);
      return CPM_ERR_ARG;
    }
  }
  if (p->elec_type < -1 || p->elec_type >= p->n_types) {
    set_error("cpm_md_create: elec_type %d outside [-1, n_types)", p->elec_type);
    return CPM_ERR_ARG;
  }
  if (!(p->lj_cut == 0.0 || (p->lj_cut > 0.0 && p->lj_cut <= c->p.rcut))) {
    set_error("cpm_md_create: lj_cut must be 0 or in (0, rcut = %g]", c->p.rcut);
    return CPM_ERR_ARG;
  }
  if (p->t_damp > 0.0 && !(p->temperature > 0.0 && std::isfinite(p->temperature) && std::isfinite(p->t_damp))) {
    set_error("cpm_md_create: a thermostat needs temperature > 0");
    return CPM_ERR_ARG;
  }
  return CPM_OK;
}

extern "C" int cpm_md_create(cpm_ctx* c, const cpm_md_params* p, int32_t n_rep, const int32_t* off_h,
                             const int32_t* type_h, const int32_t* group_h, void* stream, cpm_md** out) {
  if (out) *out = nullptr;
  if (!c || !p || !off_h || !type_h || !out) {
    set_error("cpm_md_create: null argument");
    return CPM_ERR_ARG;
  }
  CPM_TRY(md_check_params(c, p));
  if (n_rep < 1 || n_rep > c->p.max_replicas) {
    set_error("cpm_md_create: n_rep %d outside [1, %d]", n_rep, c->p.max_replicas);
    return CPM_ERR_CAPACITY;
  }
  if (off_h[0] != 0) {
    set_error("cpm_md_create: offsets[0] must be 0");
    return CPM_ERR_ARG;
  }
  for (int r = 0; r < n_rep; ++r) {
    const int cnt = off_h[r + 1] - off_h[r];
    if (cnt < 0 || cnt > c->p.max_elyt) {
      set_error("cpm_md_create: replica %d has %d sites (capacity %d)", r, cnt, c->p.max_elyt);
      return cnt < 0 ? CPM_ERR_ARG : CPM_ERR_CAPACITY;
    }
  }
  const int n = off_h[n_rep];
  const int G = p->n_groups;
  std::vector<int> slot(std::max(1, n));
  std::vector<double> ndof((size_t)n_rep * G, 0.0);
  for (int r = 0; r < n_rep; ++r) {
    for (int j = off_h[r]; j < off_h[r + 1]; ++j) {
      const int t = type_h[j], g = group_h ? group_h[j] : 0;
      if (t < 0 || t >= p->n_types || !(p->mass[t] > 0.0) || g < 0 || g >= G) {
        set_error("cpm_md_create: site %d: type %d (mass > 0 required) or group %d out of range", j, t, g);
        return CPM_ERR_ARG;
      }
      slot[j] = r * G + g;
      ndof[(size_t)r * G + g] += 3.0;
    }
  }
  std::vector<double> Qm(ndof.size(), 0.0);
  if (p->t_damp > 0.0)
    for (size_t i = 0; i < Qm.size(); ++i) Qm[i] = ndof[i] * KB_EV * p->temperature * p->t_damp * p->t_damp;

  cpm_md* m = new cpm_md();
  m->ctx = c;
  m->p = *p;
  m->nrep = n_rep;
  m->n = n;
  m->ngroups = G;
  m->nslots = n_rep * G;
  std::vector<double> mt(2 * kLjMaxTypes, 0.0);
  for (int t = 0; t < kLjMaxTypes; ++t) {
    const bool used = t < p->n_types;
    mt[t] = used && p->mass[t] > 0.0 ? 0.5 * p->dt / (p->mass[t] * MVV2E) : 0.0;
    mt[MD_HALF_M + t] = used ? 0.5 * p->mass[t] * MVV2E : 0.0;
    m->lj.sig_half[t] = used ? 0.5 * p->lj_sigma[t] : 0.0;
    m->lj.sqrt_eps[t] = used ? std::sqrt(p->lj_epsilon[t]) : 0.0;
  }
  m->lj.elec_type = p->elec_type;
  m->lj.cut = p->lj_cut;
  cudaStream_t st = (cudaStream_t)stream;
  auto fail = [&](int status) {
    md_free(m);
    return status;
  };
  const size_t ns = (size_t)m->nslots;
  const size_t n1 = (size_t)std::max(1, n);
#define MD_ALLOC(ptr, bytes)                                                         \
  do {                                                                               \
    cudaError_t e_ = cudaMalloc(&(ptr), (bytes));                                    \
    if (e_ != cudaSuccess) {                                                         \
      set_error("cpm_md_create: cudaMalloc: %s", cudaGetErrorString(e_));            \
      return fail(e_ == cudaErrorMemoryAllocation ? CPM_ERR_NOMEM : CPM_ERR_CUDA);   \
    }                                                                                \
  } while (0)
  MD_ALLOC(m->off, sizeof(int) * (n_rep + 1));
  MD_ALLOC(m->type, sizeof(int) * n1);
  MD_ALLOC(m->slot, sizeof(int) * n1);
  MD_ALLOC(m->F, sizeof(double) * 3 * n1);
  MD_ALLOC(m->e_coul, sizeof(double) * NENERGY * n_rep);
  MD_ALLOC(m->thermo, sizeof(double) * 2 * ns);
  MD_ALLOC(m->ke, sizeof(double) * (ns + 1));
  MD_ALLOC(m->kcur, sizeof(double) * ns);
  MD_ALLOC(m->s, sizeof(double) * ns);
  MD_ALLOC(m->ndof, sizeof(double) * ns);
  MD_ALLOC(m->Qm, sizeof(double) * ns);
  MD_ALLOC(m->mt, sizeof(double) * 2 * kLjMaxTypes);
#undef MD_ALLOC
  auto up = [&](void* dst, const void* src, size_t bytes) -> int {
    if (bytes == 0) return CPM_OK;
    CPM_CUDA(cudaMemcpyAsync(dst, src, bytes, cudaMemcpyHostToDevice, st));
    return CPM_OK;
  };
  int rc = CPM_OK;
  if ((rc = up(m->off, off_h, sizeof(int) * (n_rep + 1))) || (rc = up(m->type, type_h, sizeof(int) * n)) ||
      (rc = up(m->slot, slot.data(), sizeof(int) * n)) || (rc = up(m->ndof, ndof.data(), sizeof(double) * ns)) ||
      (rc = up(m->Qm, Qm.data(), sizeof(double) * ns)) || (rc = up(m->mt, mt.data(), sizeof(double) * mt.size())))
    return fail(rc);
  if (cudaMemsetAsync(m->thermo, 0, sizeof(double) * 2 * ns, st) != cudaSuccess ||
      cudaMemsetAsync(m->F, 0, sizeof(double) * 3 * n1, st) != cudaSuccess ||
      cudaMemsetAsync(m->e_coul, 0, sizeof(double) * NENERGY * n_rep, st) != cudaSuccess) {
    set_error("cpm_md_create: cudaMemsetAsync failed");
    return fail(CPM_ERR_CUDA);
  }
  if (cudaStreamSynchronize(st) != cudaSuccess) {
    set_error("cpm_md_create: stream synchronisation failed");
    return fail(CPM_ERR_CUDA);
  }
  m->lj.type = m->type;
  *out = m;
  return CPM_OK;
}

namespace {
// Sets ctx->lj for the duration of an MD call.
struct LjScope {
  cpm_ctx* c;
  LjScope(cpm_ctx* c_, const LjSetup* lj) : c(c_) { c->lj = lj; }
  ~LjScope() { c->lj = nullptr; }
};
}  // namespace

extern "C" int cpm_md_run(cpm_md* m, int32_t n_steps, double* xyzq, double* vel, const double* dpsi, double* q,
                          double* psibar, double* energy, double* force, void* stream) {
  if (!m || !xyzq || !vel || !dpsi || !q || n_steps < 0) {
    set_error("cpm_md_run: null pointer or negative step count");
    return CPM_ERR_ARG;
  }
  cpm_ctx* c = m->ctx;
  cudaStream_t st = (cudaStream_t)stream;
  cudaStreamCaptureStatus cap = cudaStreamCaptureStatusNone;
  CPM_CUDA(cudaStreamIsCapturing(st, &cap));
  const bool capturing = cap == cudaStreamCaptureStatusActive;
  if (capturing && !m->forces_valid) {
    set_error("cpm_md_run: run once outside a capture first (the forces at the start are not known)");
    return CPM_ERR_ARG;
  }
  LjScope scope(c, m->p.lj_cut > 0.0 ? &m->lj : nullptr);
  const int k = m->p.charge_every;
  const long long step0 = m->step;
  auto force_eval = [&](bool want_energy) -> int {
    double* en = want_energy ? m->e_coul : nullptr;
    if (m->step % k == 0) return cpm_step(c, m->nrep, m->off, xyzq, dpsi, q, psibar, m->F, nullptr, en, stream);
    return cpm_forces(c, m->nrep, m->off, xyzq, dpsi, q, m->F, nullptr, en, stream);
  };
  const bool thermostat = m->p.t_damp > 0.0;
  const bool want_energy = energy != nullptr;
  if (!m->forces_valid || (n_steps == 0 && want_energy)) {
    CPM_TRY(force_eval(want_energy && n_steps == 0));
    m->forces_valid = true;
  }
  const int n = m->n;
  const int nb = std::max(1, (n + 255) / 256);
  const double kT = KB_EV * m->p.temperature;
  const double dt = m->p.dt;
  const size_t kbytes = sizeof(double) * m->nslots;
  // With a thermostat each kick_ke launch ends by zeroing ke and its block counter, so only the
  // first one of the call needs them cleared; without one ke is cleared before every launch.
  MdThermo th{0, m->nslots, m->thermo, m->ndof, m->Qm, kT, dt, m->s, m->kcur,
              reinterpret_cast<unsigned int*>(m->ke + m->nslots)};
  CPM_CUDA(cudaMemsetAsync(m->ke, 0, kbytes + sizeof(double), st));
  th.mode = thermostat && n_steps > 0 ? NH_LEAD : 0;
  CPM_CUDA(launch_pdl(k_md_kick_ke, nb, 256, 0, st, n, vel, m->F, m->type, m->slot, m->mt, 0, m->ke, th));
  MD_LAUNCH(c);
  for (int i = 0; i < n_steps; ++i) {
    CPM_CUDA(launch_pdl(k_md_kick_drift, nb, 256, 0, st, n, xyzq, vel, m->F, m->type, m->slot, thermostat ? m->s : nullptr, m->mt,
                                        dt, c->p.box[0], c->p.box[1]));
    MD_LAUNCH(c);
    ++m->step;
    CPM_TRY(force_eval(want_energy && i == n_steps - 1));
    if (thermostat)
      th.mode = i == n_steps - 1 ? NH_TRAIL : (NH_TRAIL | NH_LEAD);
    else
      CPM_CUDA(cudaMemsetAsync(m->ke, 0, kbytes, st));
    CPM_CUDA(launch_pdl(k_md_kick_ke, nb, 256, 0, st, n, vel, m->F, m->type, m->slot, m->mt, 1, m->ke, th));
    MD_LAUNCH(c);
  }
  if (thermostat && n_steps > 0) {
    CPM_CUDA(launch_pdl(k_md_scale, nb, 256, 0, st, n, vel, m->slot, m->s));
    MD_LAUNCH(c);
  }
  if (want_energy) {
    CPM_CUDA(launch_pdl(k_md_energy, (m->nrep + 127) / 128, 128, 0, st, m->nrep, m->ngroups, m->e_coul, c->scal,
                                                        (thermostat && n_steps > 0) ? m->kcur : m->ke, m->thermo,
                                                        m->ndof, m->Qm, kT, thermostat ? 1 : 0, energy));
    MD_LAUNCH(c);
  }
  if (force) CPM_CUDA(cudaMemcpyAsync(force, m->F, sizeof(double) * 3 * (size_t)n, cudaMemcpyDeviceToDevice, st));
  if (capturing) m->step = step0;          // a captured call runs on replay: cpm_md_advance counts those
  return CPM_OK;
}

extern "C" int cpm_md_advance(cpm_md* m, int64_t n_steps) {
  if (!m || n_steps < 0) {
    set_error("cpm_md_advance: null handle or negative count");
    return CPM_ERR_ARG;
  }
  m->step += n_steps;
  return CPM_OK;
}

extern "C" int cpm_md_get_state(const cpm_md* m, int64_t* step, double* thermo_host, void* stream) {
  if (!m) {
    set_error("cpm_md_get_state: null handle");
    return CPM_ERR_ARG;
  }
  if (step) *step = m->step;
  if (thermo_host) {
    cudaStream_t st = (cudaStream_t)stream;
    CPM_CUDA(cudaMemcpyAsync(thermo_host, m->thermo, sizeof(double) * 2 * m->nslots, cudaMemcpyDeviceToHost, st));
    CPM_CUDA(cudaStreamSynchronize(st));
  }
  return CPM_OK;
}

extern "C" int cpm_md_set_state(cpm_md* m, int64_t step, const double* thermo_host, void* stream) {
  if (!m || step < 0) {
    set_error("cpm_md_set_state: null handle or negative step");
    return CPM_ERR_ARG;
  }
  cudaStream_t st = (cudaStream_t)stream;
  if (thermo_host) {
    CPM_CUDA(cudaMemcpyAsync(m->thermo, thermo_host, sizeof(double) * 2 * m->nslots, cudaMemcpyHostToDevice, st));
    CPM_CUDA(cudaStreamSynchronize(st));
  }
  m->step = step;
  m->forces_valid = false;
  return CPM_OK;
}

extern "C" int cpm_md_info(const cpm_md* m, int32_t* n_sites, int32_t* n_slots) {
  if (!m) {
    set_error("cpm_md_info: null handle");
    return CPM_ERR_ARG;
  }
  if (n_sites) *n_sites = m->n;
  if (n_slots) *n_slots = m->nslots;
  return CPM_OK;
}

extern "C" void cpm_md_destroy(cpm_md* m) { md_free(m); }
