/*
 * cpm.h - C ABI of the GB300 constant-potential-method (CPM) electrostatics library.
 *
 * The library computes, for fixed electrode sites carrying Gaussian charges and a mobile
 * electrolyte of point charges in a 3-D periodic orthorhombic cell, the per-timestep CPM
 * electrostatics of Tee & Searles (arXiv 2201.12963):
 *
 *   b      electrolyte-electrode vector of Eq. 3 (b = -(electrolyte potential at each electrode
 *          site); Eq. 4 reads Psi = A q - b).  The "b" of q = S(psi - b) in other texts is -b.
 *   q      electrode charges, q = S (b + dpsi v) with S the constraint-projected inverse
 *          elastance (O A^-1, Eqs. 8-9, or O_1 O A^-1, Eqs. 13-15) and v the geometry vector.
 *   F      forces on all sites, E the electrostatic energy.
 *
 * Geometry (Sec. II.B):
 *   CPM_FF       finite field (Eqs. 10-11): v = d - z/L_z, one neutrality constraint;
 *   CPM_DOUBLED  doubled cell (Eqs. 12-15): v = d, constraints on the whole cell and sub-cell 1;
 *   CPM_SLAB     slab with z padded by slab_factor and the Yeh-Berkowitz dipole term, v = d.
 * d = +1/2 on sites with side +1 and -1/2 on side -1 (Eq. 5).
 *
 * Units: lengths in Angstrom, charges in e, potentials in V, energies in eV, forces in eV/A.
 * Coulomb constant 14.3996454784 eV A / e^2.
 *
 * Conventions for every entry point below:
 *   - Return CPM_OK (0) or a negative cpm_status; no call aborts or throws across the ABI.
 *   - "_dev" pointers are device memory owned by the caller; they must stay valid until the
 *     work queued on `stream` completes.  "_host" pointers are host memory, read during the call.
 *   - `stream` is a cudaStream_t passed as void* (NULL = legacy default stream).  All device work
 *     is queued on it; the per-step calls never synchronise the host, never allocate memory and
 *     can be captured into a CUDA graph.
 *   - One context serves one stream at a time; it is not thread-safe.
 *   - Errors a kernel detects (non-finite coordinates, a site outside the cell in z) are latched
 *     in a device status word and returned by cpm_status().
 *   - Electrolyte input is replica-major: replica r owns sites offsets[r] .. offsets[r+1]-1 of
 *     xyzq (x, y, z, Q per site, float64, base address 32-byte aligned).  x, y may be unwrapped;
 *     z must lie in [0, L_z).  Each replica's electrolyte must be electrically neutral.
 */
#ifndef CPM_GB300_H
#define CPM_GB300_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct cpm_ctx cpm_ctx;

enum cpm_geometry { CPM_FF = 0, CPM_DOUBLED = 1, CPM_SLAB = 2 };

/* CPM_FP64: every kernel computes in float64.
 * CPM_MIXED: pair, B-spline and mesh work and the stored S in float32 with compensated or float64
 * accumulation; A, its Cholesky factorisation, the neutrality projection and all energy sums stay
 * float64. */
enum cpm_precision { CPM_FP64 = 0, CPM_MIXED = 1 };

/* Reciprocal part of A (cpm_params.matrix_kspace).
 * CPM_KSPACE_EWALD: the direct Ewald sum over k-vectors up to kmax_build (the converged continuum
 *   result; its cost grows with N_e^2 times the k-vector count, which is large for big cells).
 * CPM_KSPACE_MESH: the SPME mesh operator of the per-step calls, A_k = W^T Phi W (W the B-spline
 *   stencils of the electrode sites, Phi the mesh convolution with the influence function), one
 *   batched FFT convolution per electrode column.  The matrix then matches the discrete
 *   electrostatics of b, the forces and the energy exactly; it differs from the Ewald form by the
 *   mesh discretisation error. */
enum cpm_matrix_kspace { CPM_KSPACE_EWALD = 0, CPM_KSPACE_MESH = 1 };

/* Doubled-cell storage of S (cpm_params.dc_blocks; CPM_DOUBLED only).  When every sub-cell-1
 * electrode site is the z-mirror image (x, y, L_z - z) of a sub-cell-0 site, A = [[P, Q], [Q, P]] in
 * the order (sub-cell 0, images), and the constrained problem separates into two N_e/2-site
 * problems q+- = S+- (y_0 +- y_1) on the sums and differences of mirror pairs, each with one
 * neutrality constraint: two half-size factorisations and half the S bytes per step.
 *   CPM_DC_AUTO    mirror blocks when the electrode is mirror-symmetric, else the full matrix;
 *   CPM_DC_MIRROR  mirror blocks, CPM_ERR_ARG if the electrode is not mirror-symmetric;
 *   CPM_DC_FULL    always the full N_e x N_e matrix. */
enum cpm_dc_blocks { CPM_DC_AUTO = 0, CPM_DC_MIRROR = 1, CPM_DC_FULL = 2 };

enum cpm_status {
  CPM_OK = 0,
  CPM_ERR_ARG = -1,        /* invalid argument (null pointer, size, parameter out of range) */
  CPM_ERR_CUDA = -2,       /* a CUDA runtime call failed; see cpm_last_error() */
  CPM_ERR_NOT_SPD = -3,    /* Cholesky factorisation of A failed (A not positive definite) */
  CPM_ERR_NONFINITE = -4,  /* non-finite coordinate or charge seen by a kernel */
  CPM_ERR_CAPACITY = -5,   /* n_rep or a replica's site count above the build-time capacity */
  CPM_ERR_DOMAIN = -6,     /* an electrolyte site outside [0, L_z) in z */
  CPM_ERR_TIMEOUT = -7,    /* a bounded device-side wait gave up */
  CPM_ERR_LIBRARY = -8,    /* cuFFT / cuBLAS / cuSOLVER reported an error */
  CPM_ERR_NOMEM = -9       /* device allocation failed during build */
};

typedef struct {
  double box[3];        /* physical cell Lx, Ly, Lz (A); for CPM_DOUBLED Lz is the doubled length */
  double eta;           /* Gaussian width of Eq. 2 (1/A), > 0 */
  double alpha;         /* Ewald splitting parameter (1/A), 0 < alpha < eta/sqrt(2) */
  double rcut;          /* real-space cutoff (A): every periodic image within rcut is summed */
  double slab_factor;   /* CPM_SLAB: the Ewald box is (Lx, Ly, slab_factor*Lz); ignored otherwise */
  double kmax_build;    /* reciprocal cutoff for building A (1/A); <= 0 selects 2 alpha sqrt(27.6) */
  int32_t grid[3];      /* SPME mesh K1, K2, K3 (each >= 2*spme_order, K3 even) */
  int32_t spme_order;   /* cardinal B-spline order p, 3 <= p <= 8 */
  int32_t geometry;     /* enum cpm_geometry */
  int32_t precision;    /* enum cpm_precision */
  int32_t max_replicas; /* capacity: largest n_rep accepted by the per-step calls, >= 1 */
  int32_t max_elyt;     /* capacity: largest electrolyte site count of one replica, >= 1 */
  int32_t matrix_kspace;/* enum cpm_matrix_kspace */
  int32_t dc_blocks;    /* enum cpm_dc_blocks (CPM_DOUBLED only) */
} cpm_params;

/*
 * cpm_build_matrix - build the elastance A (Eq. 3) of a fixed electrode, factorise it and keep
 * the projected inverse S (Eqs. 8-9 / 13-15; precomputed once because the electrodes are fixed,
 * Sec. II.A), A^-1 C, (C^T A^-1 C)^-1 and S v, plus every workspace the per-step calls need.
 *
 *   p               parameters (copied).
 *   n_elec          number of electrode sites N_e >= 2.
 *   elec_xyz_host   [N_e*3] float64 positions (A), row-major (x, y, z).
 *   elec_side_host  [N_e] int32, +1 or -1: the electrode each site belongs to (d = +-1/2).
 *   elec_cell_host  [N_e] int32 sub-cell label 0/1 (CPM_DOUBLED only; NULL otherwise).
 *   stream          stream for the build work; the call synchronises it before returning.
 *   out             receives the new context (set to NULL on failure).
 * A is built in float64 on the GPU: real-space Gaussian-Gaussian pairs over all images within
 * rcut, the reciprocal part (direct Ewald sum up to kmax_build, or the SPME mesh operator, see
 * cpm_matrix_kspace), self terms, and for CPM_SLAB the dipole term.  A mirror-symmetric doubled
 * cell is stored as two half-size blocks (cpm_dc_blocks).  Returns CPM_ERR_ARG before any device
 * work for invalid parameters or labels and for two sites within 1e-6 A of each other (periodic
 * images included: their Gaussian-Gaussian kernel would be 0/0), CPM_ERR_NONFINITE for a non-finite
 * coordinate, CPM_ERR_NOT_SPD if a Cholesky factorisation fails, CPM_ERR_NOMEM if device memory runs
 * out.
 */
int cpm_build_matrix(const cpm_params* p, int32_t n_elec, const double* elec_xyz_host,
                     const int32_t* elec_side_host, const int32_t* elec_cell_host, void* stream,
                     cpm_ctx** out);

/*
 * Matrix images: S is the expensive part of a context (assembling A, a dense Cholesky
 * factorisation and inverse: seconds to a minute at tens of thousands of sites) and depends only
 * on the electrode and the parameters below, so it can be kept (on disk, by the caller) and a later
 * context built from it.  The paper has no counterpart (it precomputes S once per run, Sec. II.A).
 *
 * cpm_matrix_key - 64-bit FNV-1a hash of every input that determines A: box, eta, alpha, rcut, the
 *   slab factor (CPM_SLAB), kmax_build (Ewald form), geometry, matrix_kspace, dc_blocks
 *   (CPM_DOUBLED), grid and spme_order (mesh form), and the electrode arrays exactly as passed
 *   (n_elec, xyz, side, cell).  Precision, capacities and the per-step mesh of the Ewald form do not
 *   enter.  Host only; the same validation as cpm_build_matrix.
 * cpm_matrix_image - with host_out NULL, *bytes receives the image size; otherwise the context's
 *   image (a header with the key and the layout, then S or the two mirror blocks in float64 rows of
 *   the stored stride, A^-1 C, S v) is written to host_out, whose size *bytes must be at least that.
 *   Synchronous.
 * cpm_build_matrix_from_image - cpm_build_matrix without assembling or factorising A: S, A^-1 C,
 *   S v and the projection scalars come from an image made by cpm_matrix_image.  CPM_ERR_ARG when
 *   the image's key or layout does not match these inputs (a stale or foreign image is refused,
 *   never used).  Everything else (electrode stencils, cell lists, meshes, plans, workspaces, the
 *   float32 copy of S for CPM_MIXED) is built as usual.
 */
int cpm_matrix_key(const cpm_params* p, int32_t n_elec, const double* elec_xyz_host, const int32_t* elec_side_host,
                   const int32_t* elec_cell_host, uint64_t* key);
int cpm_matrix_image(const cpm_ctx* ctx, void* host_out, int64_t* bytes);
int cpm_build_matrix_from_image(const cpm_params* p, int32_t n_elec, const double* elec_xyz_host,
                                const int32_t* elec_side_host, const int32_t* elec_cell_host, const void* image_host,
                                int64_t image_bytes, void* stream, cpm_ctx** out);

/*
 * cpm_step_charges - one CPM charge update for n_rep replicas sharing the electrode (Sec. II.A,
 * "the main computational burden ... is to obtain b"): cell list, real-space b, SPME spread,
 * FFT, influence function, inverse FFT, gather at the electrode sites, S-apply and the
 * neutrality projection.
 *
 *   n_rep             1 <= n_rep <= max_replicas.
 *   elyt_offsets_dev  [n_rep+1] int32 site offsets (offsets[0] = 0).
 *   elyt_xyzq_dev     [offsets[n_rep]*4] float64 (x, y, z, Q) per electrolyte site.
 *   dpsi_dev          [n_rep] float64 potential differences (V).
 *   q_dev             [n_rep*N_e] float64 output charges (e), replica-major.
 *   b_dev             [n_rep*N_e] float64 output b (V) or NULL.
 *   psibar_dev        [n_rep*ncons] float64 output offset potentials (V) or NULL; ncons = 1, or 2
 *                     for CPM_DOUBLED (psibar, psibar_1 of Eq. 12).
 */
int cpm_step_charges(cpm_ctx* ctx, int32_t n_rep, const int32_t* elyt_offsets_dev,
                     const double* elyt_xyzq_dev, const double* dpsi_dev, double* q_dev,
                     double* b_dev, double* psibar_dev, void* stream);

/*
 * cpm_forces - forces (and optionally energies) for given electrode charges q_dev
 * [n_rep*N_e]: SPME of all charges plus real-space pair forces, with the finite-field force
 * -Q dpsi/L_z (Sec. II.B.1) or the slab dipole force.
 *
 *   f_elyt_dev   [offsets[n_rep]*3] float64 forces on the electrolyte sites (eV/A) or NULL.
 *   f_elec_dev   [n_rep*N_e*3] float64 forces on the electrode sites or NULL.
 *   energy_dev   [n_rep*4] float64 or NULL: per replica (U, H, dH/d(dpsi), Q_+).  U is the
 *                Coulomb energy of Eq. 3 (plus the slab dipole term) evaluated as the full Ewald
 *                sum of the given charges; H = U - dpsi q^T v (+ dpsi/L_z sum Q_j Z_j for CPM_FF) is
 *                the constant-potential energy whose gradient is minus the force at the
 *                constrained optimum; dH/d(dpsi) = -q^T v (+ sum Q_j Z_j / L_z for CPM_FF) is its
 *                explicit derivative; Q_+ is the total charge of the side +1 sites.
 */
int cpm_forces(cpm_ctx* ctx, int32_t n_rep, const int32_t* elyt_offsets_dev,
               const double* elyt_xyzq_dev, const double* dpsi_dev, const double* q_dev,
               double* f_elyt_dev, double* f_elec_dev, double* energy_dev, void* stream);

/* cpm_energy - energies only: cpm_forces with both force outputs NULL (energy_dev [n_rep*4] required). */
int cpm_energy(cpm_ctx* ctx, int32_t n_rep, const int32_t* elyt_offsets_dev,
               const double* elyt_xyzq_dev, const double* dpsi_dev, const double* q_dev,
               double* energy_dev, void* stream);

/*
 * cpm_step - one whole electrostatic step: cpm_step_charges followed by cpm_forces on the new
 * charges, sharing the cell list.  Outputs as above; q_dev is required, the rest may be NULL.
 * Because q is the constrained optimum here, U is assembled in closed form,
 * U = U_elyt - q^T b / 2 + dpsi q^T v / 2 (A q = b + dpsi v + C psibar, C^T q = 0), which needs no
 * electrode-electrode pair sum; it agrees with the full sum of cpm_energy to the mesh error.
 */
int cpm_step(cpm_ctx* ctx, int32_t n_rep, const int32_t* elyt_offsets_dev,
             const double* elyt_xyzq_dev, const double* dpsi_dev, double* q_dev, double* psibar_dev,
             double* f_elyt_dev, double* f_elec_dev, double* energy_dev, void* stream);

/*
 * cpm_capacitance - dQ/d(dpsi) = e_+^T S v (e/V): the charge response of all side +1 sites to the
 * potential difference (q is linear in dpsi, Eqs. 8, 11, 14).  For CPM_DOUBLED it covers the
 * positive electrodes of both sub-cells.  Host output, no device work.
 */
int cpm_capacitance(const cpm_ctx* ctx, double* dq_ddpsi_host);

/*
 * cpm_copy_matrix - copy a build-time matrix to host memory (diagnostics and tests).
 *   which = 0: S (float64, N_e x N_e row-major); 1: S v (N_e); 2: A^-1 C (N_e x ncons row-major).
 * Always in the original site order; for mirror blocks the full matrices are assembled on the host
 * from the blocks.
 */
int cpm_copy_matrix(const cpm_ctx* ctx, int32_t which, double* host_out);

/* cpm_info - sizes: n_elec, ncons, the mesh point count and the real-space cell count. */
int cpm_info(const cpm_ctx* ctx, int32_t* n_elec, int32_t* ncons, int64_t* mesh_points,
             int32_t* n_cells);

/*
 * cpm_matrix_layout - how S is stored: *mirror_blocks = 1 for the two mirror blocks of a
 * mirror-symmetric doubled cell (cpm_dc_blocks), else 0; *s_bytes = bytes of stored S the S-apply
 * streams per replica-step with the current S-apply variant (float32 for CPM_MIXED, float64 for
 * CPM_FP64, rows padded to 4; the packed upper-triangle tiles for CPM_SAPPLY_SYM and
 * CPM_SAPPLY_SYM_TMA).
 * Either pointer may be NULL.
 */
int cpm_matrix_layout(const cpm_ctx* ctx, int32_t* mirror_blocks, int64_t* s_bytes);

/*
 * cpm_pair_list_layout - the electrode-electrode force list of the frozen electrode (Sec. II.B
 * real-space sum; mixed precision builds it): *pairs = ordered pairs within r_c (periodic images
 * included), *table = distinct G vectors of the compressed form (a lattice electrode: entries of
 * 4 bytes, j | t << 16, with the table in shared memory), or 0 for the full form (16 bytes per
 * pair: G and j); *pairs = *table = 0 without a list (float64 contexts).  Either pointer may be
 * NULL.
 */
int cpm_pair_list_layout(const cpm_ctx* ctx, int64_t* pairs, int32_t* table);

/*
 * cpm_status - synchronise `stream`, then return and clear the device status word: CPM_OK, or the
 * first error a kernel latched (CPM_ERR_NONFINITE, CPM_ERR_DOMAIN, CPM_ERR_TIMEOUT).
 */
int cpm_status(cpm_ctx* ctx, void* stream);

/* Phases timed by the per-call profiler (cpm_profile_enable / cpm_profile_read). */
enum cpm_phase {
  CPM_PH_CELL_LIST = 0,   /* electrolyte binning and counting sort */
  CPM_PH_B_REAL = 1,      /* real-space Gaussian-point part of b */
  CPM_PH_B_SPREAD = 2,    /* SPME charge assignment of the electrolyte */
  CPM_PH_B_FFT = 3,       /* forward FFT, influence function, inverse FFT (charge update) */
  CPM_PH_B_GATHER = 4,    /* mesh potential at the electrode sites, b assembly */
  CPM_PH_S_APPLY = 5,     /* q = S b + dpsi S v */
  CPM_PH_PROJECT = 6,     /* neutrality projection and offsets */
  CPM_PH_F_SPREAD = 7,    /* SPME charge assignment of all charges */
  CPM_PH_F_FFT = 8,       /* forward FFT, influence function (+ energy), inverse FFT (forces) */
  CPM_PH_F_GATHER = 9,    /* mesh forces on all sites */
  CPM_PH_F_PAIR_ELYT = 10,/* real-space forces / energy, electrolyte targets */
  CPM_PH_F_PAIR_ELEC = 11,/* real-space forces / energy, electrode targets */
  CPM_PH_ENERGY = 12,     /* energy assembly */
  CPM_NPHASES = 13
};

/*
 * cpm_profile_enable - per-phase CUDA-event timing of subsequent per-step calls.  capacity > 0
 * allocates room for that many timed (phase, call) intervals and starts recording (events are
 * recorded on each call's stream around each phase); capacity = 0 stops recording and frees the
 * events.  Intervals beyond the capacity are not recorded.  Not for use during graph capture.
 */
int cpm_profile_enable(cpm_ctx* ctx, int32_t capacity);

/*
 * cpm_profile_read - synchronise the device, then write the accumulated milliseconds
 * (ms_host[CPM_NPHASES]) and interval counts (count_host[CPM_NPHASES]) of everything recorded
 * since the last read, and reset the accumulators.
 */
int cpm_profile_read(cpm_ctx* ctx, double* ms_host, int64_t* count_host);

/* cpm_counters - number of this library's kernels launched by the per-step calls of ctx so far
 * (host-side count; a CUDA graph replay of a captured call launches the same kernels again
 * without adding to it). */
int cpm_counters(const cpm_ctx* ctx, int64_t* kernel_launches);

/*
 * cpm_step_charges_static - the charge update of cpm_step_charges for a single replica, for
 * callers that must not allocate device memory while they run: code executing where cudaMalloc
 * is unavailable or forbidden (inside another library's allocator-free region, real-time loops
 * with a no-allocation policy, hosts whose memory pools are owned by someone else).  The paper
 * has no counterpart; it is a deployment convenience.
 *
 * All per-call scratch (cell list, SPME meshes, b and its float32 split, reduction slots) lives
 * in one file-scope __device__ array of CPM_STATIC_SCRATCH_BYTES bytes that every GPU loading the
 * library holds until the process exits; this call never calls cudaMalloc, cudaFree or an
 * allocating library routine.  The context (built earlier by cpm_build_matrix) supplies S, the
 * stencils and the FFT plans.  Arguments are those of cpm_step_charges with n_rep = 1:
 * elyt_offsets_dev [2], q_dev / b_dev [N_e], psibar_dev [ncons].
 *
 * - The array's device address is looked up (cudaGetSymbolAddress, with the device current) when
 *   a context is built on that device, so a context built after a cudaDeviceReset sees the
 *   array where the reloaded library put it.  On a device with no context built since the
 *   library was loaded, the first call does the lookup: make that call before any stream capture.
 * - Returns CPM_ERR_CAPACITY (see cpm_last_error) when the context's mesh, electrolyte capacity
 *   and electrode count need more scratch than CPM_STATIC_SCRATCH_BYTES.
 * - Every call shares the one array and it keeps the previous call's contents (each call clears
 *   what must start at zero): calls that overlap on the GPU — on different streams, or on
 *   different contexts of the same device — race and corrupt each other.  Serialise them.
 */
#define CPM_STATIC_SCRATCH_BYTES (32u * 1024u * 1024u)
int cpm_step_charges_static(cpm_ctx* ctx, const int32_t* elyt_offsets_dev, const double* elyt_xyzq_dev,
                            const double* dpsi_dev, double* q_dev, double* b_dev, double* psibar_dev,
                            void* stream);

/* Kernel variants of the single-replica mixed-precision S-apply (cpm_set_sapply_variant,
 * cpm_autotune):
 *   CPM_SAPPLY_ROWS    one warp per row of S, the right-hand side read through L1;
 *   CPM_SAPPLY_STREAM  one persistent CTA per SM holding the right-hand side in shared memory,
 *                      every warp streaming an equal contiguous span of S (row partial sums are
 *                      added in float64 and finished by a second kernel), 8 16-byte loads of S in
 *                      flight per lane.  Available when the right-hand side fits shared memory
 *                      (rows of at most 25,600 entries);
 *   CPM_SAPPLY_STREAM16  the same with 16 loads in flight per lane;
 *   CPM_SAPPLY_SYM     S (or each mirror block) kept as the upper triangle of 128 x 128 float32
 *                      tiles: one read of an off-diagonal tile serves its rows and, transposed, its
 *                      columns, so about half the bytes of S are streamed; each tile's row and
 *                      column sums are added into a float64 row vector with atomics.  With at
 *                      most 16 tiles per CTA (S of up to about 8,800 rows, or mirror blocks of
 *                      that size) the same kernel also forms the projection sums (exact
 *                      fixed-point sums of its float32 products) and the projection finishes the
 *                      rows; with more tiles a second kernel finishes them.  Same availability as
 *                      the streaming variants; the packed copy costs half an extra float32 S in
 *                      memory;
 *   CPM_SAPPLY_SYM_TMA the same packed tiles moved into shared memory by bulk asynchronous copies
 *                      (three 64 KB stages per CTA, all requested at the start; bounded mbarrier
 *                      waits that latch CPM_ERR_TIMEOUT), the right-hand side read per tile.
 *                      Available where CPM_SAPPLY_SYM is.
 * Batches of 8 or more replicas use the tensor-core GEMM and 2-7 replicas the row kernel whatever
 * the choice; float64 contexts always use the row kernel. */
enum cpm_sapply_variant { CPM_SAPPLY_ROWS = 0, CPM_SAPPLY_STREAM = 1, CPM_SAPPLY_STREAM16 = 2, CPM_SAPPLY_SYM = 3,
                          CPM_SAPPLY_SYM_TMA = 4 };

/* cpm_set_sapply_variant - select the S-apply variant; CPM_ERR_ARG if it is not available for
 * this context (the streaming variants need CPM_MIXED and rows of at most 25,600 entries). */
int cpm_set_sapply_variant(cpm_ctx* ctx, int32_t variant);

/* Mesh convolution of the mixed-precision path (cpm_set_fft_variant, cpm_autotune):
 *   CPM_FFT_LIBRARY  cuFFT real-to-complex / complex-to-real with a separate influence kernel;
 *   CPM_FFT_OWN      this library's float32 transform in five launches (z, y, x with the influence
 *                    function between the forward and inverse transforms, y, z), each line in
 *                    shared memory as a four-step direct transform.  Available when the x and y
 *                    mesh sizes fit the shared-memory tiles (at most 400 points).
 * Float64 contexts always use the library transform. */
enum cpm_fft_variant { CPM_FFT_LIBRARY = 0, CPM_FFT_OWN = 1 };

/* cpm_set_fft_variant - select the mesh convolution; CPM_ERR_ARG if it is not available. */
int cpm_set_fft_variant(cpm_ctx* ctx, int32_t variant);

/* Charge assignment and force interpolation of the mixed-precision path (cpm_set_mesh_variant,
 * cpm_autotune):
 *   CPM_MESH_SITES  one warp per site in input order, B-spline stencils added into the mesh with
 *                   float32 atomics and interpolated from it directly;
 *   CPM_MESH_BRICK  one block per group of 2 x 2 x 2 real-space cells of the cell-sorted sites: the
 *                   stencils of the group are accumulated in a shared-memory brick that one TMA
 *                   tensor reduction adds into a halo-padded mesh (folded onto the periodic mesh
 *                   before the transform); forces are interpolated from a brick of the padded
 *                   potential loaded by one TMA tensor copy.
 * Float64 contexts always use CPM_MESH_SITES. */
enum cpm_mesh_variant { CPM_MESH_SITES = 0, CPM_MESH_BRICK = 1 };

/* cpm_set_mesh_variant - select the charge assignment; CPM_ERR_ARG if it is not available. */
int cpm_set_mesh_variant(cpm_ctx* ctx, int32_t variant);

/*
 * cpm_set_pair_group / cpm_get_pair_group - z cells per block of the real-space pair kernels.  A
 * block computes the targets of gz consecutive cells along z (contiguous in the cell-sorted list)
 * against the sources of their joint stencil, so its setup, stencil scan and source staging serve
 * gz times the targets for (gz + 2 s) / (1 + 2 s) times the sources (s the stencil half-width), at
 * the price of more distance checks per target.  Default 1; cpm_autotune times 1 to 4.
 * CPM_ERR_ARG if gz is outside 1..8 or its stencil exceeds the kernel's tables.
 */
int cpm_set_pair_group(cpm_ctx* ctx, int32_t gz);
int cpm_get_pair_group(const cpm_ctx* ctx, int32_t* gz);

/*
 * cpm_set_wait_test - test hook for the bounded device waits (on != 0: on; default off).  The
 * only spin-waits of the library are the mbarrier waits of the tcgen05 S-apply (batched replicas,
 * mixed precision) and of the TMA brick force gather (cpm_mesh_variant brick).  Each polls a
 * bounded number of times; if it gives up it latches CPM_ERR_TIMEOUT, waits once more with the same
 * bound for the tensor-core work or copy still in flight, and leaves without using its result.
 * With the hook on, the first of those waits gives up without polling, so a call that reaches one
 * of the two kernels returns invalid results and latches CPM_ERR_TIMEOUT (read by the next call
 * or by cpm_status); turning it off restores normal calls.  It takes effect at launch, so a CUDA
 * graph keeps the setting it was captured with.  CPM_ERR_ARG for a null context.
 */
int cpm_set_wait_test(cpm_ctx* ctx, int32_t on);

/* Real-space pair kernels (the real-space part of b, the electrolyte and electrode forces, the
 * Gaussian-Gaussian energy) come in two forms:
 *   cell blocks      one block per cell (or z group of cells, cpm_set_pair_group): the sources of
 *                    the cells within r_c of the cell are staged in shared memory and shared by its
 *                    targets;
 *   warp per target  the stencil cells within r_c of the target point itself, sources read from
 *                    global memory through the caches, no block-wide staging or barriers.
 * Both compact the sources within r_c into a per-warp queue before the screened kernels, and give the
 * same results up to the order of the sums.  The variant is a mask of the target kinds that use the
 * warp form: electrode targets (real-space b, electrode forces) and electrolyte targets (electrolyte
 * forces, with the MD loop's Lennard-Jones).  CPM_PAIR_N3_ELYT (combinable with CPM_PAIR_WARP_ELEC, not
 * with CPM_PAIR_WARP_ELYT): the electrolyte forces of the mixed path by a cell kernel that applies
 * Newton's third law to the electrolyte-electrolyte pairs (one block per cell, the half stencil,
 * each pair evaluated once, the reaction added to the source with float32 atomics into a
 * cell-sorted force buffer); used where the cell kernel would be, outside an MD loop with
 * Lennard-Jones and with the site charge assignment; the same forces to float32 rounding.
 * Default CPM_PAIR_CELL; cpm_autotune times all six. */
enum cpm_pair_variant { CPM_PAIR_CELL = 0, CPM_PAIR_WARP_ELEC = 1, CPM_PAIR_WARP_ELYT = 2, CPM_PAIR_WARP = 3,
                        CPM_PAIR_N3_ELYT = 4 };
int cpm_set_pair_variant(cpm_ctx* ctx, int32_t variant);
int cpm_get_pair_variant(const cpm_ctx* ctx, int32_t* variant);

/*
 * cpm_autotune - choose the kernel variants on the given single-replica input, in stages: every
 * available S-apply variant, then with that S-apply the two mesh convolutions (cpm_fft_variant),
 * then the two charge assignments (cpm_mesh_variant), then the pair-kernel variants
 * (cpm_pair_variant) together with their z groups of 1 to 4 cells (cpm_set_pair_group).  A
 * stage captures the whole step of each candidate (the current choice among them) as a CUDA graph
 * on a private stream and replays them interleaved for 15 rounds after a warm-up round, each
 * replay started with a cold L2 cache and timed with CUDA events (direct calls when the profiler
 * is on); the smallest median wins.  Each timed call is a whole cpm_step with forces on all
 * sites, electrolyte and electrode (scratch force and energy outputs).  choice_host[3] (may be NULL) receives the kept
 * (cpm_sapply_variant, cpm_fft_variant, cpm_mesh_variant); cpm_get_pair_group and
 * cpm_get_pair_variant report the rest.
 * Allocates and frees a scratch buffer of twice the L2 size, scratch outputs, a stream and the
 * timing graphs.  The arguments are those of
 * cpm_step_charges with n_rep = 1; q_dev receives the charges.  Synchronises `stream`; not for
 * use during graph capture.  Without an available alternative it keeps the current variant.
 */
int cpm_autotune(cpm_ctx* ctx, const int32_t* elyt_offsets_dev, const double* elyt_xyzq_dev,
                 const double* dpsi_dev, double* q_dev, void* stream, int32_t* choice_host);

/*
 * cpm_density_z - the x-y averaged charge density rho(z) across the cell (Sec. II.C, Fig. 7), for
 * the potential profile.  nbins bins of width h = L_z / nbins over the Ewald box in z (slab: the
 * padded box); rho_dev [n_rep * nbins] float64 (e / A^3) is ADDED to, so repeated calls over a
 * trajectory accumulate a sum (zero it first; divide by the number of calls through `scale` of
 * cpm_potential_z).  Electrolyte point charges count in the bin of their wrapped z; each electrode
 * site's Gaussian charge (Eq. 2, width eta) is integrated over the bins it reaches.  q_dev
 * [n_rep * N_e] are the electrode charges (e.g. from cpm_step_charges).  nbins >= 4.
 */
int cpm_density_z(cpm_ctx* ctx, int32_t n_rep, const int32_t* elyt_offsets_dev, const double* elyt_xyzq_dev,
                  const double* q_dev, int32_t nbins, double* rho_dev, void* stream);

/*
 * cpm_potential_z - the potential profile psi(z) (V) from rho: the 1-D Poisson equation
 * psi'' = -rho / eps0 (Sec. II.C) with the periodic second difference on the bin centres, solved
 * exactly (two prefix sums, the same solution as inverting the finite-difference matrix), zero
 * mean.  The mean of rho (non-zero only for a non-neutral input) is removed first.  CPM_FF adds
 * the applied ramp dpsi z / L_z, so psi jumps by dpsi across the cell boundary; CPM_DOUBLED and
 * CPM_SLAB keep psi continuous.  rho is scaled by `scale` (1 / number of accumulated samples).
 * psi_dev [n_rep * nbins]; dpsi_dev [n_rep]; 4 <= nbins <= 12288.
 */
int cpm_potential_z(cpm_ctx* ctx, int32_t n_rep, int32_t nbins, const double* rho_dev, double scale,
                    const double* dpsi_dev, double* psi_dev, void* stream);

/* ---------------------------------------------------------------------------------------------
 * Molecular dynamics around the per-step calls (Appendix A: velocity-Verlet at a 2 fs step, a
 * Nose-Hoover thermostat on the electrolyte with one thermostat per doubled-cell sub-cell;
 * Appendix B: charges re-solved every 5 steps and held in between).  The electrode is frozen and
 * every electrolyte site is a point ion: a position, a charge (the w of xyzq), a mass and a
 * Lennard-Jones type.  Units: fs, amu, A, eV, K.
 *
 * One step: thermostat half step (Trotter splitting of Martyna, Tuckerman, Tobias & Klein 1996:
 * quarter-step v_xi update, velocity scaling exp(-v_xi dt/2), xi += v_xi dt/2, quarter step;
 * Q = g k_B T t_damp^2 with g = 3 N_group), v += dt/2 F/m, x += dt v (x and y wrapped into the
 * cell), forces at the new positions, v += dt/2 F/m, thermostat half step.  The step index n
 * counts force evaluations (the first one, at the starting positions, is n = 0); when n is a
 * multiple of charge_every the charges are re-solved (cpm_step), otherwise the previous charges are
 * kept (cpm_forces).  Forces are the electrostatic forces of cpm_forces plus a synthetic
 * Lennard-Jones term (Lorentz-Berthelot mixing, force-shifted at lj_cut so energy and force vanish
 * continuously there; electrolyte-electrolyte and electrolyte-electrode pairs over every periodic
 * image within lj_cut), evaluated by the same cell list as the real-space Coulomb pairs.
 * ------------------------------------------------------------------------------------------- */
#define CPM_MD_MAX_TYPES 8
#define CPM_MD_NENERGY 8   /* per replica: U, H, U_LJ, KE, E_thermostat, E_total, T (K), Q_+ */

typedef struct {
  double dt;                             /* time step (fs), > 0 */
  int32_t charge_every;                  /* k >= 1 */
  int32_t n_types;                       /* 1 .. CPM_MD_MAX_TYPES */
  double mass[CPM_MD_MAX_TYPES];         /* amu; > 0 for every type an electrolyte site uses */
  double lj_sigma[CPM_MD_MAX_TYPES];     /* A, >= 0 */
  double lj_epsilon[CPM_MD_MAX_TYPES];   /* eV, >= 0 (0: the type takes no Lennard-Jones part) */
  int32_t elec_type;                     /* Lennard-Jones type of every electrode site, -1: none */
  int32_t n_groups;                      /* thermostat groups per replica, 1 .. 4 */
  double lj_cut;                         /* A, 0 < lj_cut <= rcut; 0 switches Lennard-Jones off */
  double temperature;                    /* K, thermostat target (> 0 when t_damp > 0) */
  double t_damp;                         /* fs, Nose-Hoover damping time; <= 0: no thermostat (NVE) */
} cpm_md_params;

typedef struct cpm_md cpm_md;

/*
 * cpm_md_create - an MD integrator for n_rep replicas of the context's electrode.
 *   elyt_offsets_host [n_rep+1] int32 site offsets (the layout of every later elyt_xyzq_dev);
 *   type_host [offsets[n_rep]] int32 in [0, n_types); group_host [offsets[n_rep]] int32 thermostat
 *   group in [0, n_groups) (NULL: all 0).  Copies them; allocates forces, thermostat state and
 *   scratch (about 24 bytes per site).  Synchronises `stream`.  The thermostat state starts at
 *   xi = v_xi = 0 and the step index at 0.  CPM_ERR_ARG for invalid parameters or labels,
 *   CPM_ERR_CAPACITY when n_rep or a replica exceeds the context's capacity.
 */
int cpm_md_create(cpm_ctx* ctx, const cpm_md_params* p, int32_t n_rep, const int32_t* elyt_offsets_host,
                  const int32_t* type_host, const int32_t* group_host, void* stream, cpm_md** out);

/*
 * cpm_md_run - advance n_steps >= 0 steps.
 *   elyt_xyzq_dev [offsets[n_rep]*4] float64 positions (updated in place) and charges (read);
 *   vel_dev [offsets[n_rep]*3] float64 velocities (A/fs, updated in place); dpsi_dev [n_rep];
 *   q_dev [n_rep*N_e] electrode charges (the held charges on entry when the next force evaluation
 *   does not re-solve them; updated at every re-solve); psibar_dev [n_rep*ncons] or NULL;
 *   energy_dev [n_rep*CPM_MD_NENERGY] or NULL: at the end of the call, per replica U and H (as
 *   cpm_forces, at the last force evaluation), U_LJ, the kinetic energy, the thermostat energy
 *   sum_g (Q_g v_xi^2 / 2 + g_g k_B T xi_g), the conserved total KE + H + U_LJ + E_thermostat, the
 *   instantaneous temperature 2 KE / (g k_B) and Q_+;
 *   force_dev [offsets[n_rep]*3] or NULL: the forces (eV/A) at the final positions, electrostatic
 *   plus Lennard-Jones.
 * The first call (and the first after cpm_md_set_state) evaluates the forces at the starting
 * positions.  No allocation and no host synchronisation: a call can be captured into a CUDA graph
 * once the forces are known (a capture before that returns CPM_ERR_ARG).  A captured call does not
 * advance the step index; the caller counts replays with cpm_md_advance, and replays a captured
 * block only from step indices congruent modulo charge_every to the one it was captured at.
 * Uses the context (its cell list, workspaces and side stream) for the call's duration.
 */
int cpm_md_run(cpm_md* md, int32_t n_steps, double* elyt_xyzq_dev, double* vel_dev, const double* dpsi_dev,
               double* q_dev, double* psibar_dev, double* energy_dev, double* force_dev, void* stream);

/* cpm_md_advance - add n_steps (graph replays) to the step index. */
int cpm_md_advance(cpm_md* md, int64_t n_steps);

/*
 * cpm_md_get_state / cpm_md_set_state - checkpoint the integrator: the step index and the
 * thermostat state thermo_host [n_rep*n_groups*2] = (xi, v_xi) per (replica, group) (NULL: not
 * copied).  Positions, velocities and electrode charges are the caller's buffers.  Both synchronise
 * `stream`; set_state marks the forces unknown, so the next cpm_md_run evaluates them at the
 * current positions with the schedule's charges (re-solved when the restored index is a multiple of
 * charge_every, else the q_dev the caller restored), continuing the checkpointed trajectory.
 */
int cpm_md_get_state(const cpm_md* md, int64_t* step, double* thermo_host, void* stream);
int cpm_md_set_state(cpm_md* md, int64_t step, const double* thermo_host, void* stream);

/* cpm_md_info - electrolyte site count and number of (replica, group) thermostat slots. */
int cpm_md_info(const cpm_md* md, int32_t* n_sites, int32_t* n_slots);

/* cpm_md_destroy - free the integrator (NULL is accepted; the context is not touched). */
void cpm_md_destroy(cpm_md* md);

/* cpm_destroy - free the context and everything it owns (NULL is accepted). */
void cpm_destroy(cpm_ctx* ctx);

/* cpm_strerror - static description of a cpm_status code. */
const char* cpm_strerror(int status);

/* cpm_last_error - detail of the last failure in the calling thread ("" if none). */
const char* cpm_last_error(void);

#ifdef __cplusplus
}
#endif

#endif /* CPM_GB300_H */
