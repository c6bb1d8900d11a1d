/*
 * dmrg_gb300.h -- C ABI of the GB300 (sm_103a) two-site DMRG sigma engine.
 *
 * The library computes the Davidson sigma step sigma = H_eff psi of the
 * two-site U(1)xU(1) ab-initio DMRG sweep (arXiv 2501.18263, Sec. 2.3,
 * Eqs. Hamilton_act_nonsym and Hamilton_act_U1sym) for the Hamiltonian of
 * Eq. 1 written in the chemist convention
 *     H = sum_ij t_ij sum_s a+_is a_js
 *       + 1/2 sum_ijkl (ij|kl) sum_st a+_is a+_kt a_lt a_js,
 * i.e. the spin-independent case of Eq. 1 with v^{Eq.1}_ijkl = (ik|jl)/2.
 * Everything numerical runs in the library's CUDA kernels on the stream given
 * at creation; no entry point falls back to the CPU.
 *
 * Conventions shared by every entry point
 *   - Orbital i of the chain carries local states (Sec. 2.1)
 *       0 = empty, 1 = beta, 2 = alpha, 3 = alpha beta (= a+_alpha a+_beta |0>);
 *     Jordan-Wigner order: chain position, then alpha before beta.
 *   - A block basis is a list of (n_alpha, n_beta) sectors in ascending
 *     lexicographic order, each with a dimension; states are numbered sector
 *     by sector.  Sector tables are int32 triples (n_alpha, n_beta, dim).
 *   - An enlarged block (left block x site, or site x right block) orders each
 *     coarse sector Q by local state s = 0..3 ascending, each sub-block holding
 *     the partner block's states of sector Q - q(s) in order.
 *   - The two-site wave function at bond k (sites k, k+1 explicit) is stored as
 *     dense row-major blocks (rows: coarse sector of L' = B_k x site k, cols:
 *     coarse sector of R' = site k+1 x C_{k+2}); dmrg_layout gives the blocks.
 *   - Device pointers are CUDA device addresses valid on the handle's device;
 *     host pointers are ordinary CPU memory.  The caller owns every buffer it
 *     passes; the library owns everything it allocates and frees it in
 *     dmrg_destroy.
 *   - A handle lives on the CUDA device that was current at dmrg_build_ops.
 *     Every call on a handle (or on a batch of handles) makes that device
 *     current for its duration and restores the caller's current device before
 *     it returns; dmrg_sigma_host_noalloc instead requires the handle's device
 *     to be current.
 *
 * Errors: every call returns a dmrg_status; nothing aborts or throws across
 * the ABI.  dmrg_last_error() gives a message for the calling thread.  After
 * DMRG_ERR_CUDA or DMRG_ERR_TIMEOUT the handle is in an undefined state and
 * must be destroyed.
 */
#ifndef DMRG_GB300_H
#define DMRG_GB300_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct dmrg_handle dmrg_handle;

typedef enum {
  DMRG_OK = 0,
  DMRG_ERR_ARG = 1,        /* invalid argument or call order */
  DMRG_ERR_OOM = 2,        /* device allocation failed or over mem_cap_bytes */
  DMRG_ERR_CUDA = 3,       /* CUDA runtime error (message in dmrg_last_error) */
  DMRG_ERR_TIMEOUT = 4,    /* a bounded device-side wait gave up */
  DMRG_ERR_NOCONV = 5,     /* Davidson reached max_iter without convergence */
  DMRG_ERR_NONFINITE = 6,  /* NaN/Inf in inputs or results */
  DMRG_ERR_STATE = 7       /* handle unusable */
} dmrg_status;

/* precision of the sigma GEMMs */
enum {
  DMRG_PREC_FP64 = 0,        /* FP64 operands, FP64 accumulation */
  DMRG_PREC_MIXED_BF16 = 1   /* split BF16 operands on tcgen05, FP32 accumulation */
};

/*
 * Problem statement (Sec. 2.1: d orbitals, N electrons, integrals t and v; the
 * bond dimension D of Eq. DefinitionMPS).
 *   t      host, L*L row-major, symmetric
 *   v      host, L^4 row-major chemist (ij|kl), 8-fold symmetric
 *   order  host permutation of 0..L-1 (chain position -> orbital) or NULL
 *   D      maximal bond dimension for sweeps (dmrg_sweep may override)
 *   seed   seed of the library's own initial state and start vectors
 *   precision  DMRG_PREC_*
 *   mem_cap_bytes  soft cap on the intermediate buffers of one sigma (0 = library default)
 * The integrals are copied; the caller may free them after the call.
 */
typedef struct {
  int32_t L, n_alpha, n_beta;
  const double* t;
  const double* v;
  const int32_t* order;
  int32_t D;
  uint64_t seed;
  int32_t precision;
  uint64_t mem_cap_bytes;
} dmrg_problem;

/* Create a handle for one problem on the current CUDA device; `cuda_stream`
 * is a cudaStream_t (NULL = default stream) on which all work is ordered. */
dmrg_status dmrg_build_ops(const dmrg_problem* problem, void* cuda_stream, dmrg_handle** out);

/*
 * Load one site isometry of an MPS basis (Eq. DefinitionMPS in block-sparse
 * form, Sec. 2.3).
 *   side = 0: left-canonical site `site`, mapping B_site x site -> B_{site+1};
 *             load in order site = 0, 1, ...
 *   side = 1: right-canonical site `site`, mapping site x C_{site+1} -> C_site;
 *             load in order site = L-1, L-2, ...
 *   sectors   host int32[n_sectors*3] of the new block (n_alpha, n_beta, dim)
 *   data      host doubles: for each new sector in order, the row-major
 *             (rows x dim) isometry whose rows are the enlarged block's states
 *             of that sector (ordering above) and whose columns are orthonormal.
 */
dmrg_status dmrg_load_site(dmrg_handle* h, int32_t site, int32_t side, int32_t n_sectors,
                           const int32_t* sectors, const double* data);

/* Build all renormalised block operators needed at `bond` (from the loaded
 * isometries) and the bond's sigma plan. */
dmrg_status dmrg_prepare(dmrg_handle* h, int32_t bond);

/* Block table of the prepared bond: int64[n_blocks*7] rows
 * (QL_alpha, QL_beta, QR_alpha, QR_beta, rows, cols, element offset); the
 * pointer is library-owned and valid until the next call on the handle. */
dmrg_status dmrg_layout(dmrg_handle* h, int32_t bond, int32_t* n_blocks, const int64_t** table,
                        int64_t* psi_size);

/* sigma = H_eff psi at `bond` (device buffers of psi_size doubles). */
dmrg_status dmrg_sigma(dmrg_handle* h, int32_t bond, const double* psi_dev, double* sigma_dev);

/* sigma at an explicit precision (DMRG_PREC_*): DMRG_PREC_FP64 is available on
 * every handle; DMRG_PREC_MIXED_BF16 needs a handle created with it. */
dmrg_status dmrg_sigma_ex(dmrg_handle* h, int32_t bond, const double* psi_dev, double* sigma_dev, int32_t precision);

/* Same with host buffers: host->device copy of psi, sigma, device->host copy. */
dmrg_status dmrg_sigma_host(dmrg_handle* h, int32_t bond, const double* psi_host, double* sigma_host);

/* Allocation-free variant of dmrg_sigma_host (the paper has no counterpart;
 * this is a library convenience).  Some callers may not allocate device memory
 * while they run: a service that sized its device memory once at start-up and
 * may not grow it, or a caller whose device allocator belongs to someone else (a
 * framework's memory pool, a fixed arena) and must not be entered from here.
 * For them psi and sigma are staged in a device array built into the library
 * (32 MiB, held by every device that loads the library until the process exits)
 * instead of a buffer allocated per call.
 * Requirements and limits:
 *   - the bond must already be prepared (dmrg_prepare), which is where all of
 *     the handle's device memory is allocated; this call allocates nothing
 *     (no cudaMalloc, no cudaMallocAsync, no allocating library routine);
 *   - psi_size <= 2097152 doubles, otherwise DMRG_ERR_ARG;
 *   - the handle's device must be current.  The first call on a device looks up
 *     the array's device address (cudaGetSymbolAddress) once and keeps it.
 * The call waits for its result (device-to-host copy) before it returns; its
 * statuses are those of dmrg_sigma_host.
 * All calls share the one array and it keeps the last call's contents: calls
 * that overlap on the GPU (other threads, other handles on the same device)
 * race with each other and must be serialised by the caller. */
dmrg_status dmrg_sigma_host_noalloc(dmrg_handle* h, int32_t bond, const double* psi_host, double* sigma_host);

/* Lowest eigenpair of H_eff at `bond` by Davidson; psi_dev is the start vector
 * on entry and the normalised eigenvector on exit; *energy its Rayleigh
 * quotient (from an FP64 sigma).  tol bounds the residual 2-norm. */
dmrg_status dmrg_davidson(dmrg_handle* h, int32_t bond, double* psi_dev, double tol, int32_t max_iter,
                          double* energy, int32_t* iterations);

/* n_sweeps full two-site sweeps (Sec. 2.1: the ALS sweep over neighbouring
 * site pairs; Sec. 4.1 names its steps Diag_H, SVD, Ren_l / Ren_r, StVec):
 * left to right over bonds 0..L-3, then right to left over bonds L-2..1, each
 * step a Davidson solve at the bond followed by the density-matrix truncation
 * to at most D_schedule[s] states (host, or NULL for problem->D) and the move
 * of the wave function to the next bond.  energies[s] (host) receives the
 * Davidson energy of the last step of sweep s.  Starts from the loaded
 * right-canonical basis at bond 0 if one was loaded, otherwise from a seeded
 * basis of kept product states.  Each Davidson solve stops when the residual
 * 2-norm of the normalised Ritz vector is <= tol; on a split-BF16 handle the
 * step whose energy is reported is refined with FP64 sigmas of its Ritz
 * vector, and the other steps stop at the residual floor of the split-BF16
 * sigma (about 1e-6 |E|).  Returns DMRG_ERR_NOCONV, with the energies
 * written, when any step reached 100 iterations without either. */
dmrg_status dmrg_sweep(dmrg_handle* h, int32_t n_sweeps, const int32_t* D_schedule, double tol,
                       double* energies);

/* dmrg_sweep with options: flags bit 0 = on a split-BF16 handle, refine every
 * step with FP64 sigmas (not only the reported one); bit 1 = mode optimisation:
 * after the eigensolver at every left-to-right step, the micro-step of
 * dmrg_mode_step (the orbitals, and with them the handle's integrals, change;
 * dmrg_get_integrals returns them, dmrg_mode_log the angles and entropies);
 * bit 2 = one layer pair of swap gates (the brick-wall permutations of global
 * mode optimisation, Sec. 2.2 and Fig. 2: Walecki's construction, every pair of
 * modes adjacent once in L/2 such sweeps): the two modes of every even bond are
 * exchanged when the bond is first visited and those of every odd bond on the
 * way back (a rotation by pi/2; no eigensolver at those steps; the state is
 * truncated to D after the swap as after any step), and the energy reported for
 * a swap step is that of the last eigensolver;
 * max_iter = Davidson iteration limit per step (<= 0: 100).  Other flag bits are
 * rejected. */
dmrg_status dmrg_sweep_ex(dmrg_handle* h, int32_t n_sweeps, const int32_t* D_schedule, double tol,
                          double* energies, int32_t flags, int32_t max_iter);

/* Per-step record of the last dmrg_sweep / dmrg_sweep_ex call (library-owned
 * host tables, valid until the next call on the handle).
 *   rows: double[n_steps * 8] = (sweep, bond, direction 1 = left to right /
 *         0 = right to left, Davidson iterations, status, energy, final
 *         residual 2-norm, discarded density-matrix weight), where status is
 *         0 converged to tol, 1 stopped at the split-BF16 residual floor,
 *         2 reached max_iter, 3 subspace exhausted (no new direction);
 *   kept: int32[n_kept * 4] = (step index, n_alpha, n_beta, kept states) for
 *         every sector of the block that the step's truncation produced, in
 *         sector order (Sec. 2.1: the kept eigenvectors of the reduced density
 *         matrix define the new block basis). */
dmrg_status dmrg_sweep_log(dmrg_handle* h, int32_t* n_steps, const double** rows, int32_t* n_kept,
                           const int32_t** kept);

/* Seconds of the last dmrg_sweep call split by phase, in the categories of the
 * paper's timing breakdown (Sec. 4.1): seconds5[0] Tables (sigma plans and
 * split operands), [1] Diag_H (Davidson), [2] SVD (density matrices,
 * eigensolver, selection), [3] Ren_l / Ren_r (renormalisation and enlargement of
 * block operators), [4] StVec (wave function moved to the next bond).  Each
 * phase boundary records a timestamp on the handle's stream (no
 * synchronisation, so the host builds the next plans while the device still
 * works); a phase is the advance of the device timeline between its boundaries:
 * the device work the phase issued, plus the time the device waited for the host
 * to issue it.  The phases add up to the sweep's wall time on the device.
 * seconds5 is host memory. */
dmrg_status dmrg_sweep_phases(dmrg_handle* h, double* seconds5);

/* Adjoint of the sigma step (the differentiation form; Sec. 2.2 uses the
 * density matrices it yields for the orbital rotations c~+ = U c+ of mode
 * optimisation).  With F = <lam| H_eff(t, v) |psi> at `bond` for the handle's
 * fixed MPS basis (psi_dev, lam_dev: device, psi_size doubles in the layout of
 * dmrg_layout), the call ADDS to the device buffers
 *   g1[i*L + j]             (L^2 doubles): dF/dt_ij, symmetrised over i <-> j;
 *   g2[((i*L + j)*L + k)*L + l]  (L^4 doubles): 2 dF/dv_ijkl, symmetrised over the
 *                           eight index permutations of a real (ij|kl);
 * in the caller's orbital numbering, i.e. for symmetric t and 8-fold symmetric v
 *   F = sum_ij t_ij g1_ij + 1/2 sum_ijkl v_ijkl g2_ijkl   (F is linear in t, v).
 * For lam = psi = the normalised eigenvector, g1 is the one-particle density
 * matrix  <E_ij> = sum_s <a+_is a_js>  (symmetric) and g2 the two-particle one
 * <sum_st a+_is a+_kt a_lt a_js>  averaged over its index symmetries, so that
 * dE/dt = g1 and dE/dv = g2 / 2.  Computed by reverse mode through the sigma
 * terms, every blocking step and every renormalisation of the left and right
 * block chains (the forward operators are those the handle holds; the adjoint
 * keeps one block's and one enlarged block's adjoints at a time and cuts its
 * sigma-term intermediates under mem_cap_bytes).  FP64 throughout.  Waits for
 * the result. */
dmrg_status dmrg_sigma_backward(dmrg_handle* h, int32_t bond, const double* psi_dev, const double* lam_dev,
                                double* g1_dev, double* g2_dev);

/* Replace the integrals (host, caller's numbering, as in dmrg_problem) and drop
 * every block operator built from the old ones; the loaded or swept MPS basis
 * and the swept wave function are kept, so that dmrg_prepare / dmrg_expectation
 * / dmrg_sigma_backward then evaluate the new Hamiltonian in the same basis
 * (how a caller differentiates E(t, v) at a fixed state, e.g. through
 * torch.autograd or by finite differences). */
dmrg_status dmrg_set_integrals(dmrg_handle* h, const double* t, const double* v);

/* The wave function the last dmrg_sweep left (at the bond it stopped on, in
 * that bond's dmrg_layout): *bond, *psi_size, and a device copy into psi_dev
 * (may be NULL to query the size). */
dmrg_status dmrg_sweep_state(dmrg_handle* h, int32_t* bond, int64_t* psi_size, double* psi_dev);

/* Make psi (device, in the layout of the prepared `bond`) the handle's current
 * state: dmrg_sweep_state returns it, dmrg_mode_step rotates it, and a following
 * dmrg_sweep starts from it when `bond` is 0.  The library keeps its own copy. */
dmrg_status dmrg_set_state(dmrg_handle* h, int32_t bond, const double* psi_dev);

/* <lam| H_eff |psi> at `bond` with the FP64 sigma (device vectors; *value on
 * the host). */
dmrg_status dmrg_expectation(dmrg_handle* h, int32_t bond, const double* lam_dev, const double* psi_dev,
                             double* value);

/* Orbital gradient (Sec. 2.2: orbital rotations U = exp(kappa), kappa real
 * antisymmetric, rotating t -> U t U^T and every index of v alike): with the
 * generalised Fock matrix F_pq = sum_r t_pr g1_qr + sum_rst v_prst g2_qrst of
 * the handle's current integrals and the density matrices g1, g2 (device, as
 * dmrg_sigma_backward writes them), grad[p*L + q] = dE/dkappa_pq at kappa = 0
 * = 2 (F_qp - F_pq) (device, L^2 doubles, antisymmetric). */
dmrg_status dmrg_orbital_gradient(dmrg_handle* h, const double* g1_dev, const double* g2_dev, double* grad_dev);

/*
 * Sharded sigma (several GPUs, one problem; the paper spreads the task list of a
 * sigma step over its GPUs, Sec. 2.4 and Fig. 5): the terms of H_eff at a bond
 * are divided among the ranks, psi is replicated, each rank computes the sum of
 * its terms, and one sum of the partial sigmas over the ranks (an all-reduce)
 * gives sigma.
 *   dmrg_term_work: *n_terms and, if work != NULL, work[nu] = algorithmic flops
 *     of term nu at `bond` (terms in the library's order; the last one is the
 *     local term H_L' (x) 1).
 *   dmrg_term_partition: owner[nu] in [0, world) for n terms (host only, no
 *     device needed, deterministic: longest-work-first onto the least loaded
 *     rank, ties to the lower index / lower rank), so every rank computes the
 *     same partition on its own.
 *   dmrg_sigma_subset: sigma_dev = the FP64 sum of the terms with
 *     owner[nu] == rank (device buffers of psi_size doubles; owner host int32 of
 *     n_terms).  The sum over all ranks equals dmrg_sigma at FP64 up to the
 *     order of summation.
 */
dmrg_status dmrg_term_work(dmrg_handle* h, int32_t bond, int32_t* n_terms, int64_t* work);
dmrg_status dmrg_term_partition(int32_t n, const int64_t* work, int32_t world, int32_t* owner);
dmrg_status dmrg_sigma_subset(dmrg_handle* h, int32_t bond, const double* psi_dev, double* sigma_dev,
                              const int32_t* owner, int32_t rank);

/* Statistics of the prepared bond: int64[16] = psi_size, n_terms,
 * flops_stage1, flops_stage2 (algorithmic sigma flops), operator_bytes,
 * gemm_problems, gemm_segments, kernel launches of one FP64 sigma, then for the
 * split-BF16 plan: stage-1 tiles, stage-1 tile x K-stage count, stage-2 tiles,
 * stage-2 tile x K-stage count, X elements, BF16 plane bytes, then
 * [14] device allocations the handle has made since it was created (every
 * cudaMallocAsync of the library on the handle's behalf; calls that allocate
 * nothing leave it unchanged) and [15] the number of term chunks of one sigma
 * (terms are cut into chunks so that the stage-1 intermediates fit under
 * mem_cap_bytes). */
dmrg_status dmrg_stats(dmrg_handle* h, int64_t* out16);

/*
 * The eigensolver of the truncation step (Sec. 2.1: the kept states of a block are
 * the leading eigenvectors of its reduced density matrix, sector by sector), on
 * caller data: nmat dense symmetric FP64 matrices, matrix b of order n[b] (host
 * array, every n[b] >= 1), packed one after the other in device memory, row-major:
 * A holds sum_b n[b]^2 doubles (destroyed), Z receives the eigenvectors as columns
 * (same layout, a separate buffer), w receives the eigenvalues of each matrix in
 * ascending order (sum_b n[b] doubles, every n[b] <= 6000).  Householder
 * tridiagonalisation and divide and conquer in FP64 (leaves of at most 32 rows by
 * implicit QL), the kernels the truncation step runs.  Returns DMRG_ERR_NOCONV
 * when a leaf's QL iteration does not converge (results undefined), DMRG_ERR_ARG
 * on bad arguments.  Runs on the handle's stream and device; synchronous.
 */
dmrg_status dmrg_eigh_batch(dmrg_handle* h, int32_t nmat, const int32_t* n, double* A_dev, double* w_dev,
                            double* Z_dev);

/*
 * Mode optimisation (Sec. 2.2, Fig. 1).  A spin-independent rotation of the two
 * orbitals at the sites k, k+1 of a bond by the angle theta: the new orbitals are
 *   c~+_k = cos(theta) c+_k + sin(theta) c+_{k+1},  c~+_{k+1} = -sin(theta) c+_k + cos(theta) c+_{k+1}
 * (U = [[c, s], [-s, c]] on chain positions k, k+1), the integrals become
 * t' = U t U^T and v'_abcd = sum U_ai U_bj U_ck U_dl v_ijkl, and the wave function
 * expressed in the new orbitals gives the same energy with t', v'.
 *   dmrg_two_site_rotate: out = psi expressed in the orbitals rotated by theta at
 *     `bond` (device, psi_size doubles each, different buffers).
 *   dmrg_half_renyi: the half-Renyi entropy S_1/2 = 2 ln Tr sqrt(rho) of the cut
 *     between the two sites of `bond` (rho the reduced density matrix of
 *     B_k x site k, psi normalised inside), by the FP64 density-matrix
 *     eigensolver of the truncation.
 *   dmrg_mode_step: the micro-step on the state a sweep left: theta that
 *     minimises S_1/2 (a scan of one period, then golden-section refinement;
 *     0 when no rotation lowers it), the state rotated, the integrals rotated and
 *     every block operator rebuilt in the same basis; *s_before, *s_after (host,
 *     may be NULL) the entropies.
 *   dmrg_get_integrals: the handle's current integrals in the caller's numbering
 *     (host t: L*L, v: L^4).
 *   dmrg_mode_log: the micro-steps of the last sweep with mode optimisation,
 *     rows (sweep, bond, theta, S_1/2 before, S_1/2 after), library-owned.
 */
dmrg_status dmrg_two_site_rotate(dmrg_handle* h, int32_t bond, double theta, const double* psi_dev, double* out_dev);
dmrg_status dmrg_half_renyi(dmrg_handle* h, int32_t bond, const double* psi_dev, double* s_half);
dmrg_status dmrg_mode_step(dmrg_handle* h, double* theta, double* s_before, double* s_after);
dmrg_status dmrg_get_integrals(dmrg_handle* h, double* t, double* v);
dmrg_status dmrg_mode_log(dmrg_handle* h, int32_t* n_steps, const double** rows);

/* Code paths of the prepared bond's sigma plans (an implementation detail,
 * reported so that tests can show which paths a case exercises): int64[8] =
 * FP64 term chunks, split-BF16 term chunks, split-K parts of split-BF16 stage 2,
 * stage-1 problems with several contributing fine blocks, stage-1 gathered-row
 * problems, largest coarse L' dimension of psi, stage-2 problems spanning more
 * than one 128-row tile, number of terms. */
dmrg_status dmrg_plan_paths(dmrg_handle* h, int64_t* out8);

/* Sigma steps replayed from a captured CUDA graph since the handle was created.
 * Every prepared bond captures its sigma step (split, grouped tensor-core or
 * FP64 GEMM launches, reductions) once per precision into a CUDA graph and
 * replays it for every Davidson iteration, when the handle's stream is a created
 * (non-default) stream that is not being captured and kernel timing is off;
 * otherwise the launches are issued one by one.  Results are identical. */
dmrg_status dmrg_graph_replays(dmrg_handle* h, int64_t* replays);

/* Kernel timing with CUDA events on the handle's stream (this library's
 * kernels only).  mode = 1: reset counters and start; mode = 0: stop and write
 * out14[2c] = milliseconds and out14[2c+1] = launches for the kernel classes
 * c = 0 FP64 GEMM, 1 blocking (kron), 2 vector, 3 eigensolvers (Rayleigh-Ritz
 * Jacobi and the density-matrix Householder + QL), 4 split-BF16
 * tensor-core GEMM of sigma stage 2 (and accumulating products), 5 split /
 * pack / reduce, 6 split-BF16 tensor-core GEMM of sigma stage 1.
 * out14 may be NULL when mode = 1. */
dmrg_status dmrg_profile(dmrg_handle* h, int32_t mode, double* out14);

/*
 * Batched form (many independent problems; the grouped launch of the sigma
 * GEMMs over the block-sparse tasks of Sec. 2.4, item (c), taken across
 * problems): the split-BF16 sigma steps of n problems, each a handle prepared at
 * its bond, run as one grouped tensor-core launch per stage whose tiles are
 * sorted together by work, so that problems too small to fill the GPU alone
 * fill it together.  Each problem's result is bit-identical to dmrg_sigma on
 * its handle.
 *   dmrg_batch_create: handles[i] (created with DMRG_PREC_MIXED_BF16, all on
 *     one device and one stream, each appearing once) must be prepared at
 *     bonds[i] (host int32[n]).  The batch copies the handles' plans into one
 *     merged plan owned by the first handle.  The handles must stay prepared at
 *     those bonds while the batch is used: after dmrg_prepare on one of them
 *     (even at the same bond) or dmrg_destroy of one of them, dmrg_batch_sigma
 *     returns DMRG_ERR_STATE.  Destroying a handle first releases the batch's
 *     plans; the batch itself must still be destroyed (either order is safe).
 *   dmrg_batch_sigma: psi_dev[i], sigma_dev[i] (host arrays of n device
 *     pointers, psi_size doubles of problem i each).  use_graph = 1 captures the
 *     whole step into a CUDA graph on the first call (and whenever the buffer
 *     pointers change) and replays it; it needs a created, non-default stream
 *     and kernel timing off.  The call waits for the step to finish.
 */
typedef struct dmrg_batch dmrg_batch;
dmrg_status dmrg_batch_create(int32_t n, dmrg_handle* const* handles, const int32_t* bonds, dmrg_batch** out);
/* The same with the tile shape of the merged launches fixed (an implementation
 * parameter; the paper has no counterpart): tile_width = 0 lets
 * dmrg_batch_create's autotuner choose the tile width (MMA N) of stages 1 and 2
 * among 128 and 64 together with the order; 64 or 128 fixes it for all three
 * launches (orders still tuned); anything else is DMRG_ERR_ARG.  Every
 * width computes each element of sigma with the same products in the same
 * order. */
dmrg_status dmrg_batch_create_ex(int32_t n, dmrg_handle* const* handles, const int32_t* bonds, int32_t tile_width,
                                 dmrg_batch** out);
dmrg_status dmrg_batch_sigma(dmrg_batch* b, const double* const* psi_dev, double* const* sigma_dev,
                             int32_t use_graph);
/* Tile schedule of the batch's merged launches (an implementation parameter;
 * the paper has no counterpart), chosen at dmrg_batch_create by
 * timing every candidate on the GPU (skipped, order 0, while kernel timing is on):
 * order3[k] for k = 0 local term, 1 stage 1, 2 stage 2, with 0 = longest tile
 * first over all problems, 1 = problems in batch order with each problem's tiles
 * together, 2 = problems by decreasing work with each problem's tiles together;
 * ms9[3k + o] (host, may be NULL) = measured milliseconds of order o for stage k
 * (0 where not timed).  The order changes only the time, never the result. */
dmrg_status dmrg_batch_schedule(dmrg_batch* b, int32_t* order3, float* ms9);
/* The autotuner's full record: order3[k] and width3[k] (tile width, MMA N) chosen
 * for launch k (0 local term, 1 stage 1, 2 stage 2); ms18[6k + 2o + w] (host, may
 * be NULL) = measured milliseconds of order o at width 128 (w = 0) or 64 (w = 1),
 * 0 where not timed.  dmrg_batch_schedule's ms9 holds the times at the chosen
 * width. */
dmrg_status dmrg_batch_tuning(dmrg_batch* b, int32_t* order3, int32_t* width3, float* ms18);
void dmrg_batch_destroy(dmrg_batch* b);

void dmrg_destroy(dmrg_handle* h);

/* Thread-local message of the last failing call (empty string if none). */
const char* dmrg_last_error(void);

#ifdef __cplusplus
}
#endif

#endif /* DMRG_GB300_H */
