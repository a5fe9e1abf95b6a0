/*
 * lrt.h -- C ABI of the GB300 DMRG linear-response library.
 *
 * The library evaluates the effective-Hamiltonian sigma vector H_eff x of the
 * DMRG sweep (Nakatani, Wouters, Van Neck, Chan, "Linear response theory for
 * the density matrix renormalization group", Sec. "Time-Independent DMRG
 * Equation", Eq. dmrg) for one- and two-site wavefunctions in the
 * mixed-canonical gauge, contracted from renormalized normal and complementary
 * operator blocks (Sec. "Sweep algorithm for the projected Hamiltonian",
 * Eqs. hzero_sb and lopr1st: the "x" summation), and the block
 * renormalization O' = L^T [O x h] L that feeds it.
 *
 * Conventions shared by every entry point
 *  - Spatial orbitals 0..k-1; spin orbitals p = 2*i + sigma (alpha first);
 *    H = sum_ij h_ij E_ij + 1/2 sum_ijkl (ij|kl)(E_ij E_kl - delta_jk E_il) + e_core.
 *  - Site states |0>, |a>, |b>, |ab> = a+_a a+_b |0>; U(1)xU(1) labels (N_a, N_b).
 *  - Bond b (0..k) separates sites 0..b-1 from b..k-1; a bond sector is labelled
 *    by the electrons LEFT of the bond and has a dimension D.
 *  - Site tensors and one-site wavefunctions use the "left-fused" layout: for
 *    each sector q_r of the right bond (table order) a row-major block whose
 *    rows are the sub-blocks n = 0..3 (left sector q_r - n, skipped if absent,
 *    D(q_l) rows each) and whose D(q_r) columns are the right states.
 *    Two-site wavefunctions on sites (i, i+1): for each sector q_m of bond i+1
 *    (table order) with non-empty fusions, a row-major block with rows (n1, l)
 *    over bond i and columns (n2, r) over bond i+2.  wfn_layout() returns sizes.
 *  - All floating point is IEEE binary64 unless `precision` selects the mixed
 *    path.
 *
 * Errors: every function returns 0 on success or a negative LRT_E* code; no
 * C++ exception or abort crosses the ABI.  lrt_last_error() describes the
 * last failure of a context.
 * Ownership: host arrays passed in are copied and stay owned by the caller;
 * device buffers passed in (x, y) belong to the caller; everything the
 * library allocates is freed by lrt_destroy().
 * Threading: a context is used by one host thread at a time; all device work
 * of a context is issued on the stream given to lrt_create().
 */
#ifndef LRT_H
#define LRT_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define LRT_OK 0
#define LRT_EINVAL (-1)   /* bad argument, size or layout */
#define LRT_ENOMEM (-2)   /* device or host allocation failed */
#define LRT_ECUDA (-3)    /* a CUDA call failed */
#define LRT_ENOCONV (-4)  /* iteration limit reached; results written, residual above tolerance */
#define LRT_ETIMEOUT (-5) /* a bounded device wait expired */
#define LRT_ESTATE (-6)   /* call order: a required object has not been built */

#define LRT_FP64 0        /* all products in binary64 on the CUDA cores */
#define LRT_MIXED 1       /* split-TF32 tensor-core products, FP32 accumulation */

typedef struct lrt_ctx* lrt_t;

/* Create a context on CUDA device `device`; `cuda_stream` is a cudaStream_t
 * (NULL = legacy default stream). */
int lrt_create(lrt_t* out, int device, void* cuda_stream);
int lrt_destroy(lrt_t ctx);
/* Message of the last failure of `ctx` (or of the last lrt_create when ctx is NULL);
 * valid until the next call on the context. */
const char* lrt_last_error(lrt_t ctx);

/* Hamiltonian (the Hamiltonian of Sec. "Illustrative Applications", ab initio form).
 * h: k*k row-major one-electron integrals; eri: k^4 chemist (ij|kl) row-major, or NULL
 * when the factor B (n_factor*k*k, (ij|kl) = sum_L B[L,i,j] B[L,k,l]) is given instead;
 * eri NULL, n_factor 0 and B NULL give a one-body operator (no two-electron part, e.g. the
 * perturbation of sweep_response).  Integrals must have the 8-fold real symmetry.
 * Replaces any previous Hamiltonian and drops all renormalized blocks. */
int op_build(lrt_t ctx, int k, const double* h, const double* eri, int n_factor,
             const double* B, double e_core);

/* Matrix product state (Eqs. mps_wave_gen, mps_wave, gauge-shift).  bond_nsect[b]
 * sectors for b = 0..k; bond_sectors holds (N_a, N_b, D) triples of all bonds
 * concatenated; site_data[i] is the host pointer to site i in the left-fused layout.
 * Bond 0 must be the single sector (0,0,1) and bond k the single sector
 * (n_alpha, n_beta, 1).  Left blocks are renormalized with site_data (the
 * left-orthonormal L_i of the mixed-canonical gauge) and right blocks with
 * site_data_right (the right-orthonormal R_i, same layout), or with site_data when
 * site_data_right is NULL.  Copied to the device; drops all renormalized blocks. */
typedef struct {
  int k;
  int n_alpha;
  int n_beta;
  const int* bond_nsect;
  const int* bond_sectors;
  const double* const* site_data;
  int center;
  const double* const* site_data_right;
} lrt_mps_desc;
int mps_load(lrt_t ctx, const lrt_mps_desc* mps);

/* mps_save: the MPS the context holds now (after mps_load, sweep_gs or tda_prepare) into
 * caller-allocated host buffers, in mps_load's layout, so that mps_load of the result
 * restores it.  A query fills the sizes: call with every buffer NULL to get k, n_alpha,
 * n_beta, total_sectors and (if site_nelem is given) the doubles of every site, then
 * allocate and call again.  bond_nsect: k+1 ints; bond_sectors: 3 * total_sectors ints
 * ((N_a, N_b, D) triples, bond by bond); site_data[i] / site_data_right[i]: host buffers of
 * site_nelem[i] doubles for the left-fused site tensors (the loaded form, and the
 * right-orthonormal form when the context holds one; a NULL array or entry skips it).
 * has_right is set to 1 when the right-orthonormal form exists.  LRT_ESTATE without an MPS. */
typedef struct {
  int k, n_alpha, n_beta;
  int total_sectors;
  int has_right;
  int* bond_nsect;
  int* bond_sectors;
  int64_t* site_nelem;
  double* const* site_data;
  double* const* site_data_right;
} lrt_mps_out;
int mps_save(lrt_t ctx, lrt_mps_out* out);

/* Size in doubles of a one-site (nsite=1, sites site) or two-site (nsite=2, sites
 * site, site+1) wavefunction; block_offsets, if non-NULL, receives the start of every
 * fused block (one per right-bond sector for nsite=1, one per populated middle sector
 * for nsite=2) and must have room for the count returned in *nblocks. */
int wfn_layout(lrt_t ctx, int site, int nsite, int64_t* nelem, int* nblocks, int64_t* block_offsets);

/* Block renormalization (Eqs. gauge-shift and lopr1st/ropr1st, zeroth order):
 * dir = +1 builds the left block of bond site+1 from the left block of bond site and
 * the (left-orthonormal) tensor of `site`; dir = -1 builds the right block of bond
 * `site` from the right block of bond site+1 and the (right-orthonormal) tensor of
 * `site`.  Left block 0 and right block k are the vacuum and always exist.
 * precision LRT_FP64, or LRT_MIXED: the enlarged operators are formed in FP64 and the
 * two grouped contractions O' = L^T (E L) run as split-TF32 tensor-core products with
 * FP32 accumulation per block product (the new operators are stored in FP64). */
int renormalize(lrt_t ctx, int site, int dir, int precision);

/* sigma = H_eff x (Eq. dmrg) for `nvec` wavefunctions stored back to back in the
 * wfn_layout order: nsite = 1 uses the left block of bond `site` and the right block
 * of bond site+1; nsite = 2 uses the left block of bond `site` and the right block of
 * bond site+2.  x_dev, y_dev: device pointers of nvec * nelem doubles; must not
 * overlap. */
int sigma(lrt_t ctx, int site, int nsite, int nvec, const double* x_dev, double* y_dev,
          int precision);

/* Diagonal of H_eff (the preconditioner of Eq. error) in the same layout as sigma. */
int heff_diag(lrt_t ctx, int site, int nsite, double* d_dev);

/* Ground state by two-site DMRG sweeps (Eq. dmrg solved by Davidson at every
 * position with the diagonal preconditioner of Eq. error; decimation by the
 * eigenvectors of the reduced density matrix of each (N_a, N_b) sector, keeping the
 * M largest weights over all sectors; gauge shift and renormalization as in
 * Eq. gauge-shift).  Starts from the loaded MPS, which must be right-orthonormal
 * with the centre on site 0, and leaves the optimized MPS loaded (right-orthonormal,
 * centre on site 0).  M_schedule[s] is the bond dimension of sweep s (the last entry
 * repeats, each held for sweeps_per_M sweeps); sweeps stop when the energy of two
 * consecutive sweeps at the final M differs by less than e_tol, or after max_sweeps.
 * e0: the lowest eigenvalue of the last Davidson solve (total energy, Eh). */
typedef struct {
  int max_sweeps;
  int n_schedule;
  const int* M_schedule;
  int sweeps_per_M;
  double e_tol;
  double dav_tol;        /* Davidson residual 2-norm */
  int dav_max_iter;
  int dav_max_space;     /* <= 48 */
  double trunc_tol;      /* density-matrix weights below trunc_tol * largest are dropped */
  int onesite_sweeps;    /* then this many one-site sweeps (Eq. dmrg at one site, bond
                            dimensions fixed, gauge shifts by per-sector SVDs), which make
                            the state stationary on the one-site manifold (the reference
                            the TDA assumes); the MPS is left in the same form */
} lrt_gs_params;
int sweep_gs(lrt_t ctx, const lrt_gs_params* params, double* e0);

/* DMRG-TDA (Fig. alg:dmrgtda).  The zeroth-order state must be loaded in its
 * mixed-canonical gauge: mps_load with site_data = L0_i (left-orthonormal) and
 * site_data_right = R0_i (right-orthonormal), then tda_load with C0[i] (left-fused
 * layout, C0_i = L0_i Lambda_{i+1} = Lambda_i R0_i, Eq. gauge-shift) and lam[b], the
 * singular values of bond b concatenated sector by sector in table order.
 * sweep_tda runs the block Davidson of Fig. alg:david_gep through forward and backward
 * sweeps: Ritz rotation of the right-block objects (Eq. ritzrot2), first-order gauge
 * shifts (Eqs. gauge_fwd, gauge_bwd, left1st, right1st), site sigma (Eqs. sigv1, sigv2),
 * residual (Eq. rnorm), diagonal preconditioner (Eq. error), projection (Eq. param),
 * reduced matrices (Eqs. hleft2, sleft2) and first-order renormalization (Eqs. lopr1st,
 * ropr1st).  Outputs omega[nroots] = theta - E0 (excitation energies, ascending),
 * resid[nroots] = sum_i |Q^C r_i|^2 of the last sweep and *e0 = <Psi0|H|Psi0>.  The
 * site residual is projected by Q^C = 1 - C0 C0^T before its norm and the
 * preconditioner: at a stationary reference its C0 component <Psi0|H|Psi_mu> vanishes
 * (Eq. rnorm assumes that); elsewhere the projected sum is the residual of the
 * Rayleigh-Ritz problem on the tangent space minus Psi0, which tends to zero at
 * convergence while the unprojected one keeps that component.
 * Returns LRT_ENOCONV (results written) when max_iter is reached first. */
typedef struct {
  int max_space;      /* N, maximum number of trial vectors (0: min(48, max(8 nroots, 24))); <= 48 */
  int max_iter;
  double eps;         /* converged when sum_i |r_i^mu|^2 < eps for every root */
  double pinv_cut;    /* Lambda^-1: singular values below pinv_cut * largest are dropped */
  uint64_t seed;      /* initial trial vectors projected by Q^C: SplitMix64 Gaussians of this
                         seed, or (seed 0) at every site the unit vector on the root's rank
                         among the lowest diagonal elements of H_0 where |C0| < 1/2 */
  int precision;      /* LRT_FP64, or LRT_MIXED: the site products H_0 C run as split-TF32
                         tensor-core products until every root's sum |r|^2 is below
                         refine_tol (or two thirds of max_iter have passed), then the sweeps
                         continue in FP64 to eps (the FP64 residual correction); with
                         max_iter >= 2 the results come from FP64 sweeps.  The first-order
                         products dH C0 are FP64 in both (their operator sets are new every
                         sweep) */
  double refine_tol;  /* LRT_MIXED: switch to FP64 below this sum |r|^2 (<= 0: 1e-6) */
  int keep;           /* Ritz vectors kept when the subspace restarts (0: nroots, the deflation
                         of Fig. alg:dmrgtda); at most max_space - nroots */
  int correction;     /* LRT_CORR_SITE (0): the correction of site i is the preconditioned
                         residual of Eq. error alone.  LRT_CORR_SWEEP (1): for a root whose last
                         sum |r|^2 is below corr_tol it also takes the coupling to the
                         corrections already formed at sites < i of the same forward sweep,
                         [H_z^{L_{i-1}} x h_i x H_0^{R_i}] C0_i with the first-order left blocks
                         of the new vector z (a forward Gauss-Seidel pass over the site blocks
                         of the tangent space, whose off-diagonal overlaps vanish, Eq. sleft2);
                         far from convergence that recursion can grow along the sweep, hence
                         the gate.  The roots it converges to are the same */
  double corr_tol;    /* LRT_CORR_SWEEP gate (<= 0: 1.0) */
  double start_shift; /* > 0: the random start vectors are damped elementwise by
                         1 / (|diag(H_0^[i]) - E0| + start_shift), which weights the
                         low-lying single-site configurations (0: plain Gaussians) */
} lrt_tda_params;
enum { LRT_CORR_SITE = 0, LRT_CORR_SWEEP = 1 };
int tda_load(lrt_t ctx, const double* const* C0, const double* const* lam);
/* tda_prepare: the mixed-canonical gauge on the GPU instead of tda_load.  Takes the
 * loaded MPS with sites 1..k-1 right-orthonormal and the centre on site 0 (the state
 * sweep_gs leaves, or an MPS loaded that way), normalizes it (*norm = its norm before,
 * may be NULL) and puts every bond in its Schmidt basis by a left-to-right pass of
 * per-sector SVDs: the loaded sites become L0_i, the right-orthonormal sites R0_i,
 * and the centres C0_i and Schmidt values Lambda_b are stored as tda_load would.
 * Bond dimensions do not change; a sector with fewer fused rows than states gets
 * zero Schmidt values (dropped by pinv_cut in sweep_tda). */
int tda_prepare(lrt_t ctx, double* norm);
/* tda_stationarity: how far the loaded reference is from a stationary point of the
 * one-site MPS manifold (Eq. dmrg at every site): *grad2 = sum_i |Q^C (H_0^[i] - E0) C0_i|^2
 * with E0 = <Psi0|H|Psi0>, the squared norm of the site components of <T|H|Psi0> (zero at
 * a one-site DMRG fixed point, the reference the TDA assumes).  Needs tda_load or
 * tda_prepare first; builds the zeroth-order environments as sweep_tda does. */
int tda_stationarity(lrt_t ctx, double* grad2, double* e0);
int sweep_tda(lrt_t ctx, int nroots, const lrt_tda_params* params, double* omega, double* resid, double* e0);
/* lrt_set_wait_limit: failure detection of the tensor-core kernels.  Every pipeline wait
 * of those kernels (copies landing, products finishing, records passed between the
 * kernel's roles) gives up after a time limit, 2 s by default: the CTA raises a flag, lets
 * the copies and products it already issued finish, releases its tensor memory and
 * returns, and the call returns LRT_ETIMEOUT with the context still usable.  seconds
 * replaces that limit for this context (0 restores the default; at most 60).
 * stall_next != 0 is a test hook: in the next tensor-core launch of this context one CTA
 * first waits on a barrier that nothing completes, so that call ends through this path
 * after `seconds`; the hook clears itself with that launch.  Not part of the paper. */
int lrt_set_wait_limit(lrt_t ctx, double seconds, int stall_next);
/* sweep_tda_density: sweep_tda, and for every root mu the one-particle transition density
 * gamma[mu * k * k + p * k + q] = <Psi^mu| sum_sigma a+_{p sigma} a_{q sigma} |Psi0> over spatial
 * orbitals p, q, with Psi^mu the root's normalized tangent vector (its overall sign is
 * arbitrary) and sum_pq gamma_pq^2 the square norm that marks single-particle excitations
 * (Sec. "Qualitative understanding of DMRG-LRT excitations", Table site_excitation).  Taken
 * from the Ritz vectors of the sweep whose residuals are reported: the vector is split at
 * the centre site k/2 into one-site pieces, each contracted with the renormalized creation
 * and pair operators of its environment (FP64, dense per bond: a bond of M states costs
 * O(M^2) doubles per operator, which limits it to bond dimensions of a few thousand).
 * Arguments and status as for sweep_tda; gamma holds nroots * k * k doubles (host). */
int sweep_tda_density(lrt_t ctx, int nroots, const lrt_tda_params* params, double* omega, double* resid, double* e0,
                      double* gamma);
/* Frequency-dependent linear response at the Tamm-Dancoff level (Sec. "Time-Dependent DMRG
 * Equation and Linear Response Theory (LRT)", Eqs. pt_ext, realresp, imagresp, psi1st).
 * A one-body perturbation V = sum_pq d_pq sum_sigma a+_{p sigma} a_{q sigma} drives the
 * reference; its two first-order components X, Y in the tangent space solve, site by site,
 *   Q^C (H_0^[i] - (E0 +- omega)) C1_i = -Q^C (dH_i C0 + V_i C0)
 * (dH_i C0: the first-order products of the rest of the component, as in the TDA sigma),
 * in forward sweeps (each site solved by preconditioned MINRES, the rest fixed) with
 * backward sweeps carrying the gauge, or (LRT_RESP_SUBSPACE) as the Galerkin solution on a
 * subspace grown by one preconditioned residual per sweep.  alpha(omega) = <V Psi0|X> +
 * <V Psi0|Y>, whose poles are the TDA excitation energies; at omega = 0 it is the static
 * response.  Both forms converge below the first pole.  Between poles the component with
 * the indefinite equations converges slowly in the subspace form (diagonal preconditioner)
 * and not at all in the site iteration. */
typedef struct {
  int max_sweeps;      /* forward + backward sweeps per component (0: 40) */
  double tol;          /* sum_i |site residual|^2 at which a component stops (0: 1e-16) */
  int minres_max;      /* MINRES iterations per site solve (0: 200) */
  double minres_tol;   /* relative preconditioned residual of a site solve (0: 1e-12) */
  double pinv_cut;     /* as in lrt_tda_params (0: 1e-12) */
  int method;          /* LRT_RESP_SITE (0): the site equations solved in forward sweeps (each
                          site by MINRES, the rest fixed; converges below the first pole);
                          LRT_RESP_SUBSPACE (1): the sweep Davidson of the TDA carried to the
                          linear system (a trial vector per sweep, the Galerkin solution on the
                          subspace; its residual settles at the floor of the TDA's, so tol
                          should stay above about 1e-10) */
  int max_space;       /* LRT_RESP_SUBSPACE: trial vectors before a restart (0: 24) */
} lrt_resp_params;
#define LRT_RESP_SITE 0
#define LRT_RESP_SUBSPACE 1
/* sweep_response: ctx holds H and the reference (op_build, mps_load, tda_prepare); vctx holds
 * V as a one-body Hamiltonian (op_build with h = d, no two-electron part, e_core 0) and the
 * same MPS, also tda_prepare'd (both references must agree bit for bit, else LRT_EINVAL).
 * FP64.  Writes *alpha, resid[2] (the last sweep's sum of squared site residuals of X and of
 * Y) and sweeps[2]; omega >= 0.  LRT_EINVAL on bad arguments, LRT_ESTATE on call order. */
int sweep_response(lrt_t ctx, lrt_t vctx, double omega, const lrt_resp_params* params, double* alpha, double* resid,
                   int* sweeps);
/* lrt_sweeps: *sweeps = the number of sweeps the last sweep_gs (two-site sweeps) or
 * sweep_tda (Davidson iterations after the start sweep) on this context ran. */
int lrt_sweeps(lrt_t ctx, int* sweeps);
/* lrt_sweep_log: the wall time of every sweep of the last sweep_tda on this context (the
 * start sweep first; each time from the sweep's start to the host synchronization that
 * ends it, so it includes all its device work) and whether its H_0 site products ran on
 * the tensor cores (1) or in FP64 (0).  Writes min(cap, n) entries to seconds and mixed
 * (host arrays of cap elements; NULL allowed when cap is 0) and the number of sweeps to *n. */
int lrt_sweep_log(lrt_t ctx, int cap, double* seconds, int* mixed, int* n);
/* sweep_tda_batched: the DMRG-TDA sweeps of Fig. alg:dmrgtda for n_inst independent
 * instances, each its own context (its own Hamiltonian and reference, prepared by
 * tda_load or tda_prepare), run concurrently: host threads (at most the host's hardware
 * threads) take the instances in turn, each driving its instance's context and stream,
 * so the host-side work of the instances overlaps, and their kernels overlap on the GPU
 * when the contexts were created on different streams.  Every instance uses nroots and
 * params.  omega and resid: n_inst * nroots values, instance-major; e0: n_inst values
 * (may be NULL).  Returns LRT_OK; LRT_ENOCONV when some instance reached max_iter first
 * (all results written); else the first other error code, whose message is in that
 * instance's lrt_last_error.  The contexts must be distinct. */
int sweep_tda_batched(const lrt_t* ctxs, int n_inst, int nroots, const lrt_tda_params* params, double* omega,
                      double* resid, double* e0);

/* Read back the loaded MPS: bond tables (bond_nsect[k+1], bond_sectors[3 * total])
 * and the left-fused data of one site (host_out may be NULL to query *nelem). */
int mps_get_bonds(lrt_t ctx, int* bond_nsect, int* bond_sectors, int* total_sectors);
int mps_get_site(lrt_t ctx, int site, double* host_out, int64_t* nelem);

/* sigma_batched: y_j = H_eff^(j) x_j for n_inst independent instances, each its own
 * context (its own Hamiltonian and MPS, on the same device), in one grouped launch per
 * phase: the instances' block products are merged into one task list (FP64) or one
 * persistent tensor-core work stream (LRT_MIXED) with tiles dealt longest-first over
 * the SMs.  Instance j uses (sites[j], nsite, nvec) like sigma() and x_dev[j], y_dev[j]
 * in its wfn_layout.  The launch runs on ctxs[0]'s stream; the other contexts must be
 * idle (or use the same stream).  The merged plan is cached in ctxs[0] and rebuilt when
 * an instance's plan changes (after renormalize); from the second call with the same
 * x/y pointers on, the whole call is replayed from a captured CUDA graph.  Errors are
 * reported on ctxs[0]. */
int sigma_batched(const lrt_t* ctxs, int n_inst, const int* sites, int nsite, int nvec, const double* const* x_dev,
                  double* const* y_dev, int precision);

/* Statistics of the last sigma call: algorithmic FLOPs (2mnk summed over the
 * products of non-zero sub-blocks of the operators, zero padding excluded),
 * FLOPs issued by the kernels (fused blocks, zero sub-blocks included), bytes
 * of operator data read, kernel launches, terms of the decomposition and
 * block products. */
typedef struct {
  double flops;
  double flops_issued;
  double op_bytes;
  int launches;
  int n_terms;
  int n_products;
} lrt_sigma_stats;
int sigma_stats(lrt_t ctx, lrt_sigma_stats* out);

/* sigma_noalloc: the same H_eff x as sigma(), for callers that must not allocate
 * GPU memory -- programs whose own memory pool owns the device, loops that cannot
 * absorb the synchronization a cudaMalloc/cudaFree may cause, code where the CUDA
 * allocator may not be entered.  The paper has no counterpart; this is a service of
 * the library.
 *  - Allocates nothing: no cudaMalloc, cudaFree or allocating library routine.  The
 *    intermediates live in one static device array of LRT_NOALLOC_SCRATCH_DOUBLES
 *    doubles (32 MiB) per device, held until process exit.  The driver reserves it
 *    on a device when the library's module is first loaded there (CUDA loads modules
 *    lazily by default), which can be the first sigma_noalloc call on that device:
 *    make that first call during set-up, where the reservation is acceptable; later
 *    calls take no device memory.
 *  - Reuses the plan that a regular sigma() call with the same (site, nsite, nvec)
 *    prepared after the last renormalize(); without one it returns LRT_ESTATE.
 *    A plan whose intermediates exceed the static array is rejected with LRT_EINVAL
 *    and a message giving both sizes.
 *  - The first call on each device resolves the array's device address
 *    (cudaGetSymbolAddress); make that first call before any stream capture.
 *  - Every call shares the one array and overwrites it: calls that may overlap on
 *    the GPU (other streams, other contexts, other threads) race and must be
 *    serialized by the caller.  Nothing has to start at zero: each call writes every
 *    intermediate before reading it.
 *  - Arguments and results as for sigma() in FP64. */
#define LRT_NOALLOC_SCRATCH_DOUBLES (4 * 1024 * 1024)
#define LRT_NOALLOC_MAX_DEVICES 64
int sigma_noalloc(lrt_t ctx, int site, int nsite, int nvec, const double* x_dev, double* y_dev);

#ifdef __cplusplus
}
#endif

#endif /* LRT_H */
