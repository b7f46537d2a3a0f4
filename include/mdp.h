/*
 * mdp.h -- C ABI of the batched auxiliary-problem (AP) solves that form the columns of
 * the discrete Calderon projection P_gamma in the Method of Difference Potentials
 * (North, Tsynkov & Turkel, "Non-Iterative Domain Decomposition for the Helmholtz
 * Equation Using the Method of Difference Potentials", Sections 3.1-3.2).
 *
 * Conventions (fixed by this library; the paper is silent or garbled on them):
 *  - Grid: auxiliary rectangle with nodes (m, n), x_m = ax0 + m*h (m = 0..nx-1),
 *    y_n = ay0 + n*h (n = 0..ny-1). Grid sets M0, M+, M-, N+, N-, gamma as in Section
 *    3.2.2 (strict inequalities for M+ = M0 inside the open subdomain).
 *  - The sine transform runs along x: u = 0 on the sides x = const. Along y the AP has
 *    u = 0 (MDP_AP_DIRICHLET4) or the local Sommerfeld condition du/dn + i k u = 0,
 *    imposed at the half node between the last two node rows with O(h^4) corrections
 *    (MDP_AP_DIRX_SOMMY; Section 3.2.1, Eq. auxiliary_problem). MDP_AP_DIRX_SOMMY_PAPER
 *    takes the Sommerfeld rows as printed (Eqs. AP_bounds_right/left, rotated; the undefined
 *    u_{M-1/2} and the i k bracket's difference quotient read as the half-node mean), which
 *    are second-order accurate; the range of P_gamma, and so any coupled solution, does not
 *    depend on the AP's boundary rows.
 *  - gamma is ordered row-major in (n, m). Column c of a subdomain's block is the basis
 *    pair Psi: c = kind*4M* + (side-1)*M* + (j-1), kind 0 = Dirichlet (psi_j, 0), kind 1 =
 *    Neumann (0, psi_j), sides 1 bottom, 2 top, 3 left, 4 right, psi_j = T_{j-1}(s)
 *    (Section 3.2.4, Eq. Psi_def; Section 3.2.5, Eq. Q_construction).
 *  - Side ownership of a gamma node: smallest |rho| (signed distance to the side's line,
 *    > 0 outside), ties within 1e-9*h to the lower side index.
 *  - Complex numbers are interleaved (re, im) doubles: the layout of torch.complex128.
 *
 * Memory: every pointer passed to mdp_project_batch, mdp_project_columns, mdp_ap_adjoint
 * and mdp_ap_solve_batch is a DEVICE pointer owned by the caller, unless stated
 * otherwise. The plan owns its own tables and workspace; all its allocation happens in
 * mdp_ap_plan (and mdp_plan_update_k never reallocates), so the compute calls allocate
 * nothing. Work is enqueued on the given CUDA stream (cudaStream_t passed as void*;
 * NULL = the legacy default stream) and the calls return without synchronising.
 *
 * Errors: argument errors are returned synchronously. A failed launch returns
 * MDP_ERR_CUDA. Device-side failures set a sticky status word that mdp_plan_status reads.
 * No C++ exception crosses this boundary. A plan is not thread-safe: one caller at a time.
 */
#ifndef MDP_H
#define MDP_H

#ifdef __cplusplus
extern "C" {
#endif

typedef struct { double re, im; } mdp_c64;

typedef enum {
  MDP_OK = 0,
  MDP_ERR_ARG = 1,       /* invalid argument (sizes, geometry, kinds) */
  MDP_ERR_CUDA = 2,      /* a CUDA runtime call or launch failed */
  MDP_ERR_NOMEM = 3,     /* device or host allocation failed in mdp_ap_plan */
  MDP_ERR_SINGULAR = 4,  /* a tridiagonal pivot below tolerance (discrete AP resonance) */
  MDP_ERR_TIMEOUT = 5,   /* a bounded device wait gave up */
  MDP_ERR_STATE = 6,     /* call not valid for this plan (e.g. host-only plan) */
  MDP_ERR_BOUNDS = 7     /* an index out of its table, workspace slice or output range, found and skipped
                            by the bounds-checked build (libmdp_checked.so, MDP_CHECKED=1) */
} mdp_status;

enum { MDP_AP_DIRICHLET4 = 0, MDP_AP_DIRX_SOMMY = 1, MDP_AP_DIRX_SOMMY_PAPER = 2 };
enum { MDP_OUT_Q = 0, MDP_OUT_P = 1 };

/* Plan flags */
#define MDP_PLAN_HOST_ONLY 0x1u   /* build host tables only; no CUDA call is made */
#define MDP_PLAN_GRAPH 0x2u       /* mdp_project_batch replays a CUDA graph of its launches */
/* Subdomains that pose the same auxiliary problem up to a translation (same grid, step, k, AP,
 * M*, index sets and gamma geometry relative to the grid) share one set of tables, and
 * mdp_project_batch of the basis columns (xi == NULL, no receivers) solves each distinct
 * problem once and copies its block to the duplicates: the paper's reuse of Q for identical
 * subdomains (Section 4). User densities, receivers and the adjoint still run per subdomain
 * (on the shared tables). mdp_plan_update_k then requires equal k within each group. */
#define MDP_PLAN_DEDUPE 0x4u
/* Kernel variants (the same results to rounding; the autotuner times them): the gamma columns of
 * the middle rows by FP64 sums instead of the tensor-core contraction, and the sine transforms of
 * the dense ring and gamma rows by direct sums instead of the FFT. */
#define MDP_PLAN_FP64_COLS 0x8u
#define MDP_PLAN_DIRECT_ROWS 0x10u

/* Plan options (0 selects the default: environment MDP_TILE_COLS / MDP_WS_MB, else 256 columns
 * per work item and a 4 GiB workspace budget; 1024 points per FFT block; 2 staged rows). */
typedef struct {
  int tile_cols;              /* columns per work item (the batching tile) */
  long long workspace_bytes;  /* budget that packs work items into waves */
  int fft_block_points;       /* complex values per block of the dense-row FFT kernels: 1024, 2048 or
                                 4096 (a block takes max(1, points / (2 Nx)) columns) */
  int tri_stages;             /* table rows the per-mode sweep stages ahead in shared memory: 2 or 4 */
} mdp_plan_options;

/* One subdomain Omega_i = (x0, x1) x (y0, y1) and its auxiliary problem
 * (Section 3.2.1: AP on the enclosing rectangle; Section 3.2.4: M* basis functions per side). */
typedef struct {
  double x0, x1, y0, y1;  /* open subdomain */
  double ax0, ay0, h;     /* AP lower-left corner and grid step (the same in x and y, Section 3.1) */
  int nx, ny;             /* AP nodes along x and y */
  double k;               /* real wavenumber on Omega_i, > 0 */
  int ap_bc;              /* MDP_AP_DIRICHLET4, MDP_AP_DIRX_SOMMY or MDP_AP_DIRX_SOMMY_PAPER */
  int n_modes;            /* M* >= 1: Chebyshev modes per side; 8*M* columns */
} mdp_subdomain;

typedef struct mdp_plan mdp_plan;

/* Build a plan for n_subs subdomains: grid sets and gamma lists (Section 3.2.2), the
 * per-mode pivoted LU factors of the AP's tridiagonal systems along y (the sine transform
 * along x diagonalises Eq. aux_FD_scheme, Section 3.2.1), sine tables, the batch schedule
 * and the device workspace. Requirements per subdomain: nx, ny >= 9; the x-extent of the
 * AP equals (nx-1)*h; M+ has at least 4 nodes per direction and gamma stays at least one
 * node away from the AP boundary; k > 0; M* >= 1.
 * Returns MDP_ERR_SINGULAR if a mode's tridiagonal system is singular to working
 * precision (a Dirichlet AP at a discrete resonance). *out is owned by the caller and is
 * released with mdp_plan_destroy. With MDP_PLAN_HOST_ONLY the plan holds host tables only
 * (layout and introspection calls work; compute calls return MDP_ERR_STATE). */
mdp_status mdp_ap_plan(const mdp_subdomain *subs, int n_subs, unsigned flags, mdp_plan **out);

/* mdp_ap_plan with explicit batching options (opt may be NULL). With MDP_PLAN_GRAPH, the first
 * mdp_project_batch call for a given (xi, out, out_kind, stream) captures all its launches into
 * a CUDA graph (stream capture), later calls with the same arguments launch that graph: one
 * launch per call. Calls on the legacy default stream (NULL) are never captured; a plan keeps
 * up to 8 graphs. Per-kernel profiling (mdp_plan_profile) sees no launches in graph mode. */
mdp_status mdp_ap_plan_ex(const mdp_subdomain *subs, int n_subs, unsigned flags, const mdp_plan_options *opt,
                          mdp_plan **out);

/* Replace the wavenumbers (k[n_subs], host array, each > 0 and finite, else MDP_ERR_ARG) and
 * refactor every sine mode in place (Section 3.2.1: the per-mode tridiagonal systems of the
 * separable AP; same grids, no reallocation). On a device plan the factorisation runs on the
 * GPU, on cuda_stream (NULL: the legacy default stream): the pivoted LU of each mode, its
 * dT/dk rows and the projection's condensed sweep table are rebuilt in the device tables. The
 * call returns when they are done; MDP_ERR_SINGULAR if a mode of the new k is singular (the
 * tables are then unusable until a successful update). Host-only plans factor on the host.
 * mdp_plan_update_k is mdp_plan_update_k_stream on the legacy default stream. */
mdp_status mdp_plan_update_k(mdp_plan *p, const double *k);
mdp_status mdp_plan_update_k_stream(mdp_plan *p, const double *k, void *cuda_stream);

/* The same refactorisation without waiting for it, so that it overlaps work already queued on
 * other streams (a sweep over k: the factorisation for the next k runs while the projection of
 * the current one does). A device plan keeps a second table set (allocated by the first call,
 * as large as the first): the new tables are built into the set no queued call is reading, on
 * cuda_stream, after the compute calls that last read that set; calls made after this one, on
 * any stream, wait for the new tables and use them. The call returns at once (it may wait on the
 * host for the upload of two calls earlier). A singular mode sets the sticky status word
 * (mdp_plan_status: MDP_ERR_SINGULAR) instead of being returned. Host-only plans: as
 * mdp_plan_update_k. */
mdp_status mdp_plan_update_k_async(mdp_plan *p, const double *k, void *cuda_stream);

/* leader[i] (host array of n_subs ints): the subdomain whose tables (and, for basis columns,
 * computed block) subdomain i shares; i itself unless MDP_PLAN_DEDUPE found an earlier
 * identical subdomain. */
mdp_status mdp_plan_leaders(const mdp_plan *p, int *leader);

/* Layout of subdomain `sub` (host values): |gamma|, its 8*M* columns, the element offset
 * of its block in the output of mdp_project_batch, and a host pointer (owned by the plan,
 * valid until destroy) to |gamma| pairs (n, m) of the gamma nodes in row-major order. Any
 * output pointer may be NULL. */
mdp_status mdp_plan_layout(const mdp_plan *p, int sub, int *gamma_size, int *n_cols,
                           long long *out_offset, const int **gamma_nm);

/* Total complex elements of the output of mdp_project_batch: sum over subdomains of
 * |gamma_i| * 8 M*_i. */
long long mdp_plan_output_size(const mdp_plan *p);

/* Projection columns of every subdomain (Section 3.2.2, Eqs. Potential_def, def_Pgamma;
 * Section 3.2.5, Eq. Q_construction):
 *   xi == NULL : the densities are the extended basis functions xi_c = Ex^(H) Psi_c
 *                (Section 3.2.3, Eq. general_extension with f = 0; Section 3.2.4);
 *   xi != NULL : user densities on gamma, complex, in the layout of `out`.
 * out_kind MDP_OUT_Q writes (P_gamma - I) xi_c = -Tr G^(h)(L^(h) w|_{M+});
 * MDP_OUT_P writes P_gamma xi_c = xi_c - Tr G^(h)(L^(h) w|_{M+}).
 * out (device, complex, mdp_plan_output_size elements): per subdomain in plan order a
 * column-major block [8 M*][|gamma|]. xi and out must not overlap. */
mdp_status mdp_project_batch(mdp_plan *p, const mdp_c64 *xi, mdp_c64 *out, int out_kind,
                             void *cuda_stream);

/* The same for columns [col0, col0 + ncols) of subdomain `sub` only: the per-column
 * (unbatched) path. xi (may be NULL) and out point to the first of those columns, each
 * column |gamma| complex values, consecutive. */
mdp_status mdp_project_columns(mdp_plan *p, int sub, int col0, int ncols, const mdp_c64 *xi,
                               mdp_c64 *out, int out_kind, void *cuda_stream);

/* Adjoint of mdp_project_batch for a real loss with cotangent cot = dLoss/d conj(out)
 * (layout of out):
 *   grad_xi[c] = (P_gamma - I)^H cot[c]  (MDP_OUT_Q) or P_gamma^H cot[c] (MDP_OUT_P),
 *                computed with the conjugate-transposed AP solve G^H (may be NULL; only
 *                meaningful for user densities);
 *   grad_k[i] += dLoss/dk_i = Re sum_c <cot_c, d out_c / d k_i>, including the
 *                k-dependence of L^(h), of the AP rows and, for basis densities, of Ex^(H)
 *                (may be NULL; device array of n_subs doubles, accumulated, not zeroed).
 * xi is the forward call's density argument (NULL = basis densities). */
mdp_status mdp_ap_adjoint(mdp_plan *p, const mdp_c64 *xi, const mdp_c64 *cot, mdp_c64 *grad_xi,
                          double *grad_k, int out_kind, void *cuda_stream);

/* Full-grid AP solves of subdomain `sub`: u = G^(h) g (adjoint = 0) or u = (G^(h))^H g
 * (adjoint = 1), for nrhs right-hand sides. g and u are device arrays [nrhs][ny][nx]
 * complex (row-major grids); only the values of g on M0 are read, and u is written on
 * every node (0 at Dirichlet nodes). (Section 3.2.1: u = G^(h) g.) */
mdp_status mdp_ap_solve_batch(mdp_plan *p, int sub, int nrhs, const mdp_c64 *g, mdp_c64 *u,
                              int adjoint, void *cuda_stream);

/* Difference potential on the whole grid (Eq. Potential_def; the reconstruction of the solution
 * inside a subdomain from its boundary density, Section 3.5): u = w - G^(h) (L^(h) w)|M+ with
 * w = xi on gamma and 0 elsewhere, for ncols densities of subdomain `sub`. xi: device
 * [ncols][|gamma|] (gamma order of mdp_plan_layout); u: device [ncols][ny][nx], written on every
 * node (on N+ it is P_N+ xi; u and xi must not overlap). Uses the plan's workspace: calls on one
 * plan must not overlap in time. */
mdp_status mdp_potential(mdp_plan *p, int sub, int ncols, const mdp_c64 *xi, mdp_c64 *u, void *cuda_stream);

/* The terms a source f adds to subdomain `sub` (Delta u + k^2 u = f; Sections 3.2.1, 3.2.3,
 * 3.2.5): the right-hand side of its system Q c = F (Eq. linear_system_equations),
 *   F = (I - P_gamma) Ex^(I) f - Tr G^(h) (B^(h) f)|M+,
 * and the source's part of the solution (Eq. potential_solution with xi = Ex^(H) + Ex^(I) f),
 *   u = P_N+ Ex^(I) f + G^(h) (B^(h) f)|M+ on every node of the grid.
 * f: device [ny][nx], the source at every node of the auxiliary grid (B^(h) f, Eq. rhs_g, is
 * applied on M+, where it uses f on N+). src4: device [|gamma|][4], at the foot point of every
 * gamma node on its owner side (mdp_plan_gamma_geometry): f, its derivative along the outward
 * normal, its second normal and second tangential derivatives (Ex^(I) f, Eqs. extension_split,
 * cartesian_extension). F: device [|gamma|]; u: device [ny][nx] (must not overlap f). Uses the
 * plan's workspace (MDP_ERR_NOMEM if it is too small for one column and two grid-sized
 * scratch arrays). */
mdp_status mdp_source_terms(mdp_plan *p, int sub, const mdp_c64 *f, const mdp_c64 *src4, mdp_c64 *F, mdp_c64 *u,
                            void *cuda_stream);

/* Householder QR of a dense complex matrix (the least-squares step of the coupled subdomain
 * system, Section 3.5 steps 2(b)-(c)). A: device, column-major, m rows, n + nrhs columns,
 * leading dimension lda >= m; 1 <= n <= m. Factors the first n columns in place (R in the upper
 * triangle with a real diagonal, the reflectors H_k = I - tau_k v_k v_k^H below the diagonal
 * with v_k(k) = 1 implied) and applies Q^H to the nrhs columns after them; tau: device [n]. The
 * least-squares solution of A(:, 0:n) x = b is then R^{-1} (Q^H b)(0:n) (mdp_triangular_solve).
 * work: device, mdp_householder_qr_work_ints(1) caller-owned ints, zeroed by the call itself on
 * cuda_stream (reflector counters, then a status word and an abort flag): after the stream has
 * finished, work[batch] is MDP_OK, or MDP_ERR_TIMEOUT if a bounded wait of the kernel gave up
 * (the output is then incomplete). One cooperative launch (all CTAs resident: the call fails
 * with MDP_ERR_CUDA if the device cannot take it); no allocation. Calls that share `work` must
 * not overlap in time. */
long long mdp_householder_qr_work_ints(int batch);
mdp_status mdp_householder_qr(int m, int n, int nrhs, mdp_c64 *A, long long lda, mdp_c64 *tau, int *work,
                              void *cuda_stream);

/* mdp_householder_qr of `batch` matrices of the same shape at A + b*stride (stride >=
 * lda * (n + nrhs)); tau: device [batch][n]; work: mdp_householder_qr_work_ints(batch) ints,
 * the status word at work[batch]. Used for the first stage of the structured least squares: one
 * QR per subdomain's rows (those touch only that subdomain's unknowns), then one of the stacked
 * triangular factors. All matrices are factored in the one launch. */
mdp_status mdp_householder_qr_batched(int batch, int m, int n, int nrhs, mdp_c64 *A, long long lda,
                                      long long stride, mdp_c64 *tau, int *work, void *cuda_stream);

/* Triangular solve with the R of mdp_householder_qr (Section 3.5 step 2(c): c = R^{-1} Q^H F, and
 * the R^{-H} of the least squares' derivative). R: device, column-major n x n with leading
 * dimension ldr >= n; only the upper triangle (row <= column) is read, so the QR's output
 * buffer is passed as it is. conj_trans = 0 solves R X = B, 1 solves R^H X = B. B: device,
 * column-major n x nrhs (ldb >= n), overwritten by X. The diagonal must be nonzero (no check: a
 * zero pivot gives inf/NaN). n * 16 bytes must fit in one CTA's shared memory (n <= 14848),
 * else MDP_ERR_ARG. Enqueued on cuda_stream; no allocation. */
mdp_status mdp_triangular_solve(int n, int nrhs, const mdp_c64 *R, long long ldr, int conj_trans, mdp_c64 *B,
                                long long ldb, void *cuda_stream);

/* C = op(A) op(B), or C += op(A) op(B) if accumulate != 0, for the small dense products of the
 * coupled system's assembly (Sections 3.3-3.5: Q times a coefficient vector, the Chebyshev
 * transform of boundary data, the receiver values). op(A) is m x k with element (i, l) at
 * A[i*rsa + l*csa], conjugated if conja != 0; op(B) is k x n with (l, j) at B[l*rsb + j*csb],
 * conjugated if conjb != 0; C(i, j) at C[i*rsc + j*csc] (C must not overlap A or B). Strides in
 * elements, any sign or order (transposes are strides). Each element sums its k products in
 * order: the result does not depend on the launch. m <= 1048560. Enqueued on cuda_stream. */
mdp_status mdp_complex_matmul(int m, int n, int k, const mdp_c64 *A, long long rsa, long long csa, int conja,
                              const mdp_c64 *B, long long rsb, long long csb, int conjb, mdp_c64 *C,
                              long long rsc, long long csc, int accumulate, void *cuda_stream);

/* The extended basis densities xi_c = Ex Psi_c on gamma (Sections 3.2.3-3.2.4: the Taylor
 * extension of the Chebyshev basis function of column c, zero on the nodes owned by other
 * sides) for columns col0 .. col0+ncols-1 of subdomain `sub`: out device [ncols][|gamma|]
 * (real values stored complex). A DD solution's density on gamma is the combination of these
 * columns with its coefficients. Uses the plan's workspace. */
mdp_status mdp_basis_densities(mdp_plan *p, int sub, int col0, int ncols, mdp_c64 *out, void *cuda_stream);

/* The full-grid solve of mdp_ap_solve_batch without a plan and without any device
 * allocation, for callers that cannot call cudaMalloc (an allocator-free runtime, or a caller
 * that owns every device byte). The paper has no counterpart: this is an interface choice.
 * `sub` (host) describes one subdomain; g and u are caller-owned device arrays
 * [nrhs][ny][nx] with the meaning of mdp_ap_solve_batch (u may equal g). Each call recomputes
 * the per-mode factors on the host and copies them, with the descriptor, into a fixed scratch
 * array of mdp_ap_solve_noalloc_limit_bytes() bytes (32 MiB) that lives in device memory for
 * the lifetime of the process on every device that loads the library (only the tables the solve
 * reads: the factor rows, the sine table and the pivot flags); the mode-space buffer uses the
 * rest of it, in chunks of right-hand sides. Grids whose tables plus one right-hand side do not
 * fit return MDP_ERR_ARG (a 641^2 grid fits, 27 right-hand sides per chunk at 257^2; a 705^2
 * grid does not). The copies come from pageable host memory, so each call
 * waits on the host until the work already queued on `cuda_stream` has finished. The call
 * cannot be captured into a CUDA graph: on a capturing stream it returns MDP_ERR_STATE and
 * enqueues nothing. The first call on a device looks up the array's device address
 * (cudaGetSymbolAddress). All calls share the one array: calls whose work overlaps on the
 * GPU (different streams, or different host threads) race and must be serialised by the
 * caller. Nothing needs zeroing between calls: every call overwrites what it reads. */
mdp_status mdp_ap_solve_noalloc(const mdp_subdomain *sub, int nrhs, const mdp_c64 *g, mdp_c64 *u,
                                int adjoint, void *cuda_stream);
long long mdp_ap_solve_noalloc_limit_bytes(void);

/* Receiver rows (for reconstruction of the solution inside subdomains, Section 3.2.2, Eq.
 * potential_solution_homo: u = P_N+ xi_gamma). rows[i] is the AP grid row n of subdomain i,
 * nlo+1 <= n <= nhi-1 (strictly inside the gamma ring), or -1 for none (host array of n_subs).
 * The receivers of subdomain i are the nodes (n, m), m = mlo+1 .. mhi-1 (not on gamma, where
 * w = 0, so P_N+ xi = -G^(h) L^(h) w there). Uploads a small descriptor array; allocates nothing
 * and synchronises the device. */
mdp_status mdp_plan_set_receivers(mdp_plan *p, const int *rows);

/* Receiver layout of subdomain `sub` (host): grid row (or -1), first node m, number of nodes
 * per column, and the element offset of its block [8M*][count] in the receiver output. */
mdp_status mdp_plan_receiver_layout(const mdp_plan *p, int sub, int *row, int *m_first, int *count,
                                    long long *offset);
long long mdp_plan_receiver_size(const mdp_plan *p);

/* mdp_project_batch that also writes the difference potential P_N+ xi_c at the receivers into
 * out_rec (device, mdp_plan_receiver_size complex elements; NULL = none). */
mdp_status mdp_project_batch_rec(mdp_plan *p, const mdp_c64 *xi, mdp_c64 *out, mdp_c64 *out_rec,
                                 int out_kind, void *cuda_stream);

/* mdp_ap_adjoint with an additional cotangent on the receiver output (cot_rec, layout of
 * out_rec; NULL = none): grad_xi and grad_k then include the receivers' contribution. */
mdp_status mdp_ap_adjoint_rec(mdp_plan *p, const mdp_c64 *xi, const mdp_c64 *cot, const mdp_c64 *cot_rec,
                              mdp_c64 *grad_xi, double *grad_k, int out_kind, void *cuda_stream);

/* Synchronise the plan's device, return and clear the sticky device status word. */
mdp_status mdp_plan_status(mdp_plan *p);

void mdp_plan_destroy(mdp_plan *p);

const char *mdp_status_string(mdp_status s);

/* ---- Host introspection (no device work; valid for host-only plans) ---- */

/* Gamma geometry of subdomain `sub` into caller host arrays of |gamma| entries: owner side
 * (1..4), signed distance rho (> 0 outside Omega) and side parameter s in [-1, 1]. */
mdp_status mdp_plan_gamma_geometry(const mdp_plan *p, int sub, int *owner, double *rho, double *s);

/* Solve one mode's tridiagonal system T_q x = b (adjoint = 0) or T_q^H x = b (adjoint = 1)
 * on the host with the plan's stored factors, q = 1..nx-2. b and x are host arrays over the
 * y unknowns (ny values for the Sommerfeld APs, n = 0..ny-1; ny-2 values for
 * MDP_AP_DIRICHLET4, n = 1..ny-2). A grid function sin(pi q m/(nx-1)) b(n) on M0 is mapped
 * by G^(h) to sin(pi q m/(nx-1)) x(n). */
mdp_status mdp_host_mode_solve(const mdp_plan *p, int sub, int q, int adjoint, const mdp_c64 *b,
                               mdp_c64 *x);

#ifdef __cplusplus
}
#endif
#endif /* MDP_H */
