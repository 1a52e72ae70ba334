/* rsx.h — C ABI of librsx: real-space exact exchange on one GB300 (sm_103a).
 *
 * Method: Panta & Strubbe, "Implementation of time-dependent Hartree-Fock in real
 * space", arXiv 2405.01522.
 *   Eq. 2 (Sec. 2)       exchange action  (Vx psi_p)(r) = -sum_j phi_j(r) int phi_j(r') psi_p(r') / |r - r'| dr'
 *   Sec. 3.1             the integral solved as a Poisson problem for rho = phi_j psi_p
 *   Eqs. 11-13 (Sec 3.1) ACE: W = Vx Phi, M = <Phi, W>, -M = L L^T, zeta = W L^-T, V^ACE = -zeta zeta^T
 *   Eqs. 6-7 (Sec. 2)    Tamm-Dancoff coupling (ia|jb) and A = diag(de) + delta_M K - K_d
 *
 * Discretisation (the paper does not fix one; this is the library's reading):
 *   grid point (z, y, x) at r = ((x - nx/2) h, (y - ny/2) h, (z - nz/2) h); orbitals are
 *   zero outside the box.  The potential of a density is V(r) = h^3 sum_r' rho(r') g(r - r')
 *   with g(d) = 1/(h |d|) and g(0) = C0/h, C0 = 3 ln(2 + sqrt 3) - pi/2 (cell average of
 *   1/r).  It is evaluated exactly (up to rounding) by FFT on the box padded to 2n per
 *   axis.  Inner products are <f, g> = h^3 sum_r f(r) g(r).
 *
 * Conventions for every call:
 *   - Array arguments are DEVICE pointers owned by the caller, contiguous, layout
 *     [orbital][z][y][x] (x fastest), element type double (RSX_FP64 context) or float
 *     (RSX_FP32 context).  Matrices (M, K, omega, X) are always double.
 *   - Work is enqueued on `stream` (a cudaStream_t; NULL = legacy default stream) and
 *     the call returns without synchronising.  Device-side failures found later
 *     (a non positive definite ACE matrix, a wait that timed out) are reported by
 *     rsx_sync_status.
 *   - Return value: RSX_OK or an error code; rsx_last_error gives a message.  No call
 *     exits, aborts or falls back to a CPU path.
 *   - The library owns only its workspace (kernel table, twiddles, FFT intermediates,
 *     panels), allocated in rsx_create or grown by the calls; it never frees or keeps
 *     caller memory.  One context per stream; contexts share no state.
 *   - Supported box edges: 16, 24, 32, 40, 48, 56, 64, 80, 96, 112 (padded 2n = 16 A
 *     with A in {2,3,4,5,6,7,8,10,12,14}); nz must equal ny, nx may differ.
 */
#ifndef RSX_H
#define RSX_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct rsx_ctx rsx_ctx;

enum {
  RSX_OK = 0,
  RSX_EINVAL = 1,         /* bad size, null pointer, unsupported aliasing */
  RSX_ENOMEM = 2,         /* device allocation failed or workspace limit exceeded */
  RSX_ECUDA = 3,          /* a CUDA runtime call failed (message in rsx_last_error) */
  RSX_ENOTPD = 4,         /* -M not positive definite in the ACE Cholesky (deferred) */
  RSX_ETIMEOUT = 5,       /* a bounded device wait gave up (deferred) */
  RSX_EUNSUPPORTED = 6,   /* box edge or mode not supported */
  RSX_EBOUNDS = 7         /* bounds-checked build only: an FFT-pass index left its array
                             (the access was skipped; deferred to rsx_sync_status) */
};

enum { RSX_FP64 = 0, RSX_FP32 = 1 };

/* Create a context for box (nz, ny, nx) with spacing h (bohr) on `device`.
 * Builds the kernel spectrum table (h^3 / N_pad times the DFT of g on the padded grid)
 * and the FFT twiddles on the device; synchronises the device once.
 * precision: RSX_FP64 or RSX_FP32 (element type of every orbital array).
 * Errors: RSX_EINVAL (null ctx, h <= 0), RSX_EUNSUPPORTED (edge), RSX_ENOMEM, RSX_ECUDA. */
int rsx_create(rsx_ctx** ctx, int nz, int ny, int nx, double h, int precision, int device);

/* Free the context and its workspace (synchronises the device).  NULL is a no-op. */
int rsx_destroy(rsx_ctx* ctx);

/* Message of the last failing call on this context ("" if none).  Valid until the next call. */
const char* rsx_last_error(const rsx_ctx* ctx);

/* Limit (bytes) on the FFT-intermediate workspace; calls split their pair batch to stay
 * within it.  Default: 40% of the device memory free at rsx_create, at most 64 GiB. */
int rsx_set_workspace_limit(rsx_ctx* ctx, size_t bytes);

/* Tuning knobs of the pair-solve path (performance only: the results stay bitwise
 * identical under every knob except p2_lanes, which changes the rounding order of the
 * line transforms, both splits being equally accurate).
 *   p2_threads     threads per CTA of the y/z transform pass: 256, 384 (FP32) or 512; a
 *                  size is used only where its line scratch and the work plane fit in
 *                  shared memory (else 256)
 *   chunk_outputs  output orbitals per exchange chunk (0 = as many as the workspace holds)
 *   p1_group       x-pass block order: 0 pair-major, G > 0 pairs fastest in groups of G
 *   p2_global      1: the y/z pass keeps its work plane in a global (L2-resident) scratch
 *                  slice per CTA even where shared memory would hold it; 0: shared memory
 *                  whenever it fits
 *   p2_lanes       radix split of the y/z line transforms, M = 2n points per line: 16 (16
 *                  lanes x A: A-point DFTs in registers, then 16-point DFTs across lanes)
 *                  or 8 (8 lanes x 2A: 2A-point DFTs, then 8-point DFTs; FP32 with
 *                  shared-memory plane and A = M / 16 in {4, 8, 12}, i.e. edges 32, 64, 96;
 *                  elsewhere the 16-lane split runs) */
typedef struct rsx_tuning {
  int p2_threads;
  int chunk_outputs;
  int p1_group;
  int p2_global;
  int p2_lanes;
} rsx_tuning;
int rsx_get_tuning(rsx_ctx* ctx, rsx_tuning* out);
/* Errors: RSX_EINVAL (null, or a knob outside the values above). */
int rsx_set_tuning_ex(rsx_ctx* ctx, const rsx_tuning* t);
/* Autotuner (the paper has no counterpart; a performance knob).  Times the exchange
 * apply for nocc x npsi pairs on synthetic device data under candidate knobs, by
 * coordinate descent from the current ones: pass-2 CTA size x plane staging x line split
 * (16 or 8 lanes), then the pass-1 block order (0, 4, 16, 64, all), then output orbitals
 * per chunk (1, 2, 4, all);
 * applies the fastest to the context.  With a non-empty cache_path the result is appended
 * to that text file, keyed by box, precision, nocc, npsi, SM count and device name, and a
 * later call with the same key applies it without timing.  chosen (may be NULL) receives
 * the knobs, best_ms the best time (-1 if taken from the cache).  Synchronises the device.
 * Errors: RSX_EINVAL, RSX_ENOMEM. */
int rsx_autotune_ex(rsx_ctx* ctx, int nocc, int npsi, const char* cache_path, rsx_tuning* chosen, double* best_ms);
/* The same, returning only two of the knobs (p2_threads, chunk_outputs). */
int rsx_autotune(rsx_ctx* ctx, int nocc, int npsi, const char* cache_path, int* p2_threads, int* chunk_outputs,
                 double* best_ms);
/* Set p2_threads and chunk_outputs, keeping the other knobs. */
int rsx_set_tuning(rsx_ctx* ctx, int p2_threads, int chunk_outputs);

/* Pair densities rho_q = a_i * b_k (Sec. 3.1: the density whose potential Eq. 2 needs),
 * q = i * nb + k.  a: [na][N], b: [nb][N], rho: [na * nb][N] (must not alias a or b).
 * Errors: RSX_EINVAL. */
int rsx_build_pair_densities(rsx_ctx* ctx, const void* a, int na, const void* b, int nb, void* rho,
                             void* stream);

/* Exact-exchange action of Eq. 2: out_p = Vx[phi] psi_p = -sum_j phi_j V[phi_j psi_p],
 * for p < npsi, j < nocc; nocc * npsi pair Poisson solves.
 * phi: [nocc][N], psi: [npsi][N], out: [npsi][N] (must not alias phi or psi).
 * Errors: RSX_EINVAL (nocc < 1, npsi < 1, null, aliasing), RSX_ENOMEM. */
int rsx_exchange_apply(rsx_ctx* ctx, const void* phi, int nocc, const void* psi, int npsi, void* out,
                       void* stream);

/* Isolated-boundary potential of one density (Sec. 3.1, the Poisson solve behind Eq. 2):
 * V(r) = h^3 sum_r' rho(r') g(r - r') with the kernel of the pair solves.  Used for the
 * Hartree potential of the SCF loop.  rho, V: [N] (must not alias).  Errors: RSX_EINVAL. */
int rsx_poisson(rsx_ctx* ctx, const void* rho, void* V, void* stream);

/* Allocation-free variant of rsx_exchange_apply (the paper has no counterpart; this is
 * a deployment aid).  For callers that must not allocate device memory once running --
 * e.g. a program whose device memory is owned by its own pool allocator sized at
 * start-up, or a latency-sensitive loop that cannot take cudaFree's implicit device
 * synchronisation when a workspace is regrown.  Same result as rsx_exchange_apply (same
 * kernels, one output orbital at a time).
 * Scratch: a fixed 64 MiB device array inside the library, held by every GPU that loads
 * its module until process exit; requires nocc * (nx + 1) * nz * ny * 2 * element size
 * <= 64 MiB (else RSX_EINVAL, nothing launched) and a box whose y/z pass fits in shared
 * memory (FP32 edges <= 112, FP64 <= 64; else RSX_EUNSUPPORTED).
 * Set-up: the FIRST call on a device looks up the array's address (cudaGetSymbolAddress);
 * under lazy module loading (the CUDA default) that lookup, and the first launch of each
 * FFT pass kernel, make the driver load their modules, which maps the 64 MiB array and
 * the kernels' code -- the first call can therefore allocate driver memory.  Create the
 * context and make one call on each device at start-up, before any stream capture; every
 * later call performs no cudaMalloc/cudaFree and calls no allocating routine.  The cached
 * address is valid until process exit (a cudaDeviceReset invalidates it: restart the
 * process).  The caller's current device is restored before the call returns.
 * All calls share the array and it keeps the last call's contents (nothing in it needs
 * to start at zero); calls that overlap on the GPU race and must be serialised. */
int rsx_exchange_apply_noalloc(rsx_ctx* ctx, const void* phi, int nocc, const void* psi, int npsi, void* out,
                               void* stream);

/* ACE projectors of Eqs. 11-12 from the orbitals phi (nocc <= 64):
 * W = Vx[phi] phi (nocc (nocc + 1) / 2 solves, rho_ij = rho_ji), M_kl = <phi_k, W_l>
 * symmetrised (FP64), -M = L L^T by FP64 Cholesky on the device, xi = L^-1 W.
 * phi: [nocc][N]; xi: [nocc][N] (must not alias phi); M_out: device double [nocc][nocc]
 * receiving the symmetrised M, or NULL.
 * Errors: RSX_EINVAL, RSX_ENOMEM; RSX_ENOTPD deferred to rsx_sync_status. */
int rsx_ace_build(rsx_ctx* ctx, const void* phi, int nocc, void* xi, double* M_out, void* stream);

/* The two steps of the ACE build after W (Eqs. 11-12), for callers that assemble W and M
 * themselves (e.g. ranks that each hold a block of W's rows, see the sharded driver):
 * rsx_gram: C[i][j] = h^3 <a_i, b_j> (device double [na][nb], na * nb <= 4096; FP64
 *   accumulation of FP32 or FP64 products).
 * rsx_ace_factor: M (device double [nocc][nocc]) is symmetrised in place, -M = L L^T by
 *   the FP64 Cholesky, xi = L^-1 W ([nocc][N]; xi may equal W).  RSX_ENOTPD deferred to
 *   rsx_sync_status.  Errors: RSX_EINVAL. */
int rsx_gram(rsx_ctx* ctx, const void* a, int na, const void* b, int nb, double* C, void* stream);
int rsx_ace_factor(rsx_ctx* ctx, double* M, const void* W, int nocc, void* xi, void* stream);

/* ACE action of Eq. 13: out_p = -sum_k xi_k <xi_k, psi_p>.  nxi * npsi <= 4096.
 * xi: [nxi][N], psi: [npsi][N], out: [npsi][N]; out may equal psi (in place), must not alias xi.
 * Errors: RSX_EINVAL. */
int rsx_ace_apply(rsx_ctx* ctx, const void* xi, int nxi, const void* psi, int npsi, void* out, void* stream);

/* Tamm-Dancoff coupling K_{ia,jb} = (ia|jb) (Eqs. 6-7) for transitions t = i * nvirt + a:
 * K = (h^6 / N_pad) sum_G w_G ghat(G) Re[conj R_t(G) R_s(G)], R_t the DFT of the padded
 * rho_t = phi_i phi_a, w_G = 1 at kx = 0, Mx/2 and 2 otherwise.  FP32 context: spectra in
 * FP32, split into bf16 hi + lo and contracted on the tensor cores (hi.hi + hi.lo + lo.hi,
 * FP32 accumulation, FP64 reduction); FP64 context: FP64 throughout.
 * phi_occ: [nocc][N], phi_virt: [nvirt][N], K: device double [nt][nt], nt = nocc * nvirt <= 4096.
 * Errors: RSX_EINVAL, RSX_ENOMEM. */
int rsx_casida_K(rsx_ctx* ctx, const void* phi_occ, int nocc, const void* phi_virt, int nvirt, double* K,
                 void* stream);

/* Spin-polarised (UHF) coupling, Eqs. 4-5 in spin orbitals: K_{ia,jb} = (ia|jb) over the
 * alpha transitions t = i * nvirt_a + a followed by the beta ones, nta + ntb <= 4096: every
 * spin block of the Coulomb-type term, from one split-BF16 panel in an FP32 context (the
 * plain FP64 form otherwise).  nocc_b or nvirt_b may be 0 (no beta transitions).
 * occ_*: [nocc_*][N], virt_*: [nvirt_*][N]; K: device double [nt][nt].
 * Errors: RSX_EINVAL, RSX_ENOMEM, RSX_EUNSUPPORTED. */
int rsx_casida_K_uhf(rsx_ctx* ctx, const void* occ_a, int nocc_a, const void* virt_a, int nvirt_a, const void* occ_b,
                     int nocc_b, const void* virt_b, int nvirt_b, double* K, void* stream);

/* Coulomb term K_d[ia,jb] = (ab|ji) = <phi_a phi_b, V[phi_j phi_i]> of Eq. 7.
 * Same arguments and layout as rsx_casida_K. */
int rsx_casida_Kd(rsx_ctx* ctx, const void* phi_occ, int nocc, const void* phi_virt, int nvirt, double* Kd,
                  void* stream);

/* Lowest nroots eigenpairs of A = diag(eps_a - eps_i) + delta_M K - K_d (Eq. 7, TDA),
 * FP64 on the device (Householder tridiagonalisation, bisection, inverse iteration).
 * eps_occ: [nocc], eps_virt: [nvirt], K and Kd: [nt][nt] device doubles (Kd may be NULL);
 * omega: [nroots] ascending (Hartree); X: [nroots][nt] eigenvectors or NULL.
 * Errors: RSX_EINVAL (nroots < 1 or > nt, nt > 4096). */
int rsx_casida_solve(rsx_ctx* ctx, const double* eps_occ, int nocc, const double* eps_virt, int nvirt,
                     const double* K, const double* Kd, double delta_M, int nroots, double* omega, double* X,
                     void* stream);
/* Lowest nroots eigenpairs of the spin-polarised TDA matrix
 * A = diag(eps_a - eps_i per spin) + K - blockdiag(K_d alpha, K_d beta) (Eqs. 4-5; the
 * exchange-type term (ij|ab) only couples transitions of one spin), with K from
 * rsx_casida_K_uhf and K_d per spin from rsx_casida_Kd (either may be NULL).
 * eps: device doubles; omega: [nroots] ascending (Hartree); X: [nroots][nt] or NULL.
 * Errors: RSX_EINVAL, RSX_ENOMEM. */
int rsx_casida_solve_uhf(rsx_ctx* ctx, const double* eps_occ_a, int nocc_a, const double* eps_virt_a, int nvirt_a,
                         const double* eps_occ_b, int nocc_b, const double* eps_virt_b, int nvirt_b, const double* K,
                         const double* Kd_a, const double* Kd_b, int nroots, double* omega, double* X, void* stream);

/* Full (non-Tamm-Dancoff) RHF linear response, Eqs. 3-5 with real orbitals, in the
 * half-size symmetric form: A = diag(eps_a - eps_i) + delta_M K - K_d (Eq. 7),
 * B[ia,jb] = delta_M (ia|bj) - (ib|aj) = delta_M K[ia,jb] - K[ib,ja];
 * A - B = L L^T (FP64 blocked Cholesky), M = L^T (A + B) L, M z = omega^2 z,
 * X + Y = omega^{-1/2} L z (normalised so that X^T X - Y^T Y = 1).  Arguments as
 * rsx_casida_solve; XpY: [nroots][nt] or NULL.  Deferred errors (rsx_sync_status):
 * RSX_ENOTPD when A - B is not positive definite or an omega^2 <= 0 (an unstable ground
 * state). */
int rsx_casida_solve_full(rsx_ctx* ctx, const double* eps_occ, int nocc, const double* eps_virt, int nvirt,
                          const double* K, const double* Kd, double delta_M, int nroots, double* omega,
                          double* XpY, void* stream);

/* Single-particle dipole matrix elements entering Eq. 8:
 * dip[d][i * nvirt + a] = <i|r_d|a> = h^3 sum_r phi_i(r) r_d phi_a(r), d = x, y, z, with
 * r = ((x - nx/2) h, (y - ny/2) h, (z - nz/2) h) at grid point (z, y, x).
 * phi_occ [nocc][N], phi_virt [nvirt][N] in the context precision; dip: [3][nocc * nvirt]
 * device doubles.  Errors: RSX_EINVAL (nocc * nvirt > 4096). */
int rsx_casida_dipoles(rsx_ctx* ctx, const void* phi_occ, int nocc, const void* phi_virt, int nvirt, double* dip,
                       void* stream);

/* Oscillator strengths, Eqs. 8-9 in atomic units (no spin factor, as written):
 * d_k = sum_t X[k][t] dip[:, t], f_k = 2/3 omega_k |d_k|^2.  omega [nroots],
 * X [nroots][nt] (TDA eigenvectors or X + Y of rsx_casida_solve_full), dip [3][nt],
 * f [nroots]: device doubles. */
int rsx_casida_oscillator(rsx_ctx* ctx, const double* omega, const double* X, int nroots, int nt, const double* dip,
                          double* f, void* stream);

/* Strength function, Eq. 10 broadened by a Lorentzian of half-width gamma (Hartree):
 * S[j] = sum_k f_k gamma / (pi ((grid[j] - omega_k)^2 + gamma^2)).  Device doubles. */
int rsx_strength_function(rsx_ctx* ctx, const double* omega, const double* f, int nroots, double gamma,
                          const double* grid, int ngrid, double* S, void* stream);

/* ---- Uneven batch of independent molecules (under one captured CUDA graph).  For every
 * molecule m (cubic box of edge edges[m] in {48, 64, 80, 96, 112}, spacing h,
 * nocc[m] <= 32 orbitals, FP32):
 *   W_m  = Vx[phi_m] phi_m   (Eq. 2 with psi = phi; nocc(nocc+1)/2 pair solves)
 *   xi_m = ACE projectors of Eqs. 11-12 (M_m, -M_m = L L^T in FP64, xi_m = L^-1 W_m).
 * The molecules are grouped by edge; each FFT pass runs as one launch per edge over all
 * pairs of that edge's molecules (device lists of each pair's orbitals and each output's
 * orbital set), then the ACE Gram and L^-1 W per molecule and one FP64 Cholesky kernel for
 * all.  rsx_batch_create builds the kernel tables of every distinct edge and allocates
 * all pair intermediates.  rsx_batch_bind takes host arrays of nmol device pointers
 * (phi[m]: [nocc][edge^3], W[m], xi[m] same shape, not aliasing) and may be called again
 * with new arrays.  rsx_batch_run records the launches into a CUDA graph on its first
 * call after a bind and replays the graph afterwards.
 * rsx_batch_sync_status synchronises and reports deferred errors (RSX_ENOTPD).
 * Errors: RSX_EINVAL, RSX_EUNSUPPORTED (edge), RSX_ENOMEM, RSX_ECUDA. */
typedef struct rsx_batch rsx_batch;
int rsx_batch_create(rsx_batch** batch, int nmol, const int* edges, const int* nocc, double h, int device);
int rsx_batch_bind(rsx_batch* batch, const void* const* phi, void* const* W, void* const* xi);
int rsx_batch_run(rsx_batch* batch, void* stream);
int rsx_batch_sync_status(rsx_batch* batch, void* stream);
const char* rsx_batch_last_error(const rsx_batch* batch);
int rsx_batch_destroy(rsx_batch* batch);

/* ---- Plain block eigensolver and learned preconditioner (the paper's eigensolvers are
 * CG and preconditioned Lanczos, Sec. 3.1; the preconditioners and the network are not in
 * the paper).  H = -1/2 Lap + V with the fourth-order finite-difference Laplacian and
 * zero boundary values, on an n^3 box of spacing h, FP32 orbitals.
 * rsx_eig_create: V device [n^3] (kept by pointer), vscale multiplies V in the network's
 *   second input channel, nband <= 21 bands.
 * rsx_eig_init: starting orbitals psi0 [nband][n^3] (device), Rayleigh-Ritz on them.
 * rsx_eig_step: one block step: residual R = H Psi - Psi theta, W = (K + T)^-1 R by
 *   jacobi_sweeps damped-Jacobi sweeps (K = -1/2 Lap, T the orbital kinetic energy), plus
 *   the network's directions |R| net(R/|R|, vscale V) when net is not NULL; Rayleigh-Ritz
 *   on [Psi, W]; theta_host[nband] receives the Ritz values.  Synchronises the stream.
 * rsx_eig_orbitals / rsx_eig_residual copy the current orbitals / last residual out. */
typedef struct rsx_eig rsx_eig;
typedef struct rsx_net rsx_net;
int rsx_eig_create(rsx_eig** eig, int n, double h, const float* V, float vscale, int nband, int device);
int rsx_eig_init(rsx_eig* eig, const float* psi0, void* stream);
int rsx_eig_step(rsx_eig* eig, rsx_net* net, int jacobi_sweeps, double* theta_host, void* stream);
int rsx_eig_orbitals(rsx_eig* eig, float* psi_out, void* stream);
int rsx_eig_residual(rsx_eig* eig, float* r_out, void* stream);
/* Energy of the current orbitals evaluated in FP64: the orbitals (FP32) are widened to
 * double, H = -1/2 Lap_FD4 + V (times the mask) is applied in double, S = <Psi, Psi> and
 * Hs = <Psi, H Psi> are summed in double and energy = trace(S^-1 Hs) (the Rayleigh-Ritz sum
 * of the block, a variational upper bound on the sum of the lowest nband eigenvalues),
 * written to energy_host.  Resolves energy differences far below the FP32 Ritz values'
 * noise (used to measure convergence to 1e-6 Ha).  Synchronises the stream.
 * Errors: RSX_EINVAL (before rsx_eig_init), RSX_EUNSUPPORTED (an exchange term is set),
 * RSX_ENOMEM (2 nband n^3 doubles of workspace, allocated on the first call). */
int rsx_eig_energy64(rsx_eig* eig, double* energy_host, void* stream);
const char* rsx_eig_last_error(const rsx_eig* eig);
int rsx_eig_destroy(rsx_eig* eig);
/* Non-local exchange term added to H (Sec. 3.1): mode 0 none; 1 the ACE operator
 * -sum_k xi_k <xi_k, .> of Eq. 13 with projectors src [count][n^3] (16 ceil(count/16)
 * 4 nband <= 4096); 2 the exact exchange Vx[src] of Eq. 2 with orbitals src [count][n^3],
 * through ctx (an FP32 context on the same box).  src (and ctx) are kept by pointer.
 * Takes effect at the next rsx_eig_step or rsx_eig_refresh.  Errors: RSX_EINVAL, RSX_ENOMEM. */
int rsx_eig_set_exchange(rsx_eig* eig, rsx_ctx* ctx, const float* src, int count, int mode);
/* Spherical domain (Sec. 3.4: a sphere with zero boundary values): H restricted to the
 * points where mask is 1 (device float [n^3] of 0 / 1, kept by pointer; NULL = the whole
 * box).  The next rsx_eig_init zeroes the starting orbitals outside it.  Errors: RSX_EINVAL. */
int rsx_eig_set_mask(rsx_eig* eig, const float* mask);
/* H has changed (V's contents or the exchange term): recompute H Psi, Rayleigh-Ritz on the
 * current orbitals, drop the previous search direction; theta_host[nband] or NULL.
 * Synchronises the stream. */
int rsx_eig_refresh(rsx_eig* eig, double* theta_host, void* stream);

/* ---- Closed-shell Hartree-Fock SCF (Sec. 3.1-3.2; the rest of Sec. 3 builds on it).
 * rho = 2 sum_i phi_i^2 over nocc orbitals (N_e = 2 nocc); Fock operator
 * F = -1/2 Lap_FD4 + V_ext + V_H[rho_in] + Vx, Vx from the orbitals entering the iteration,
 * either as ACE (use_ace != 0: Eqs. 11-13 built once per iteration) or exact (Eq. 2 in
 * every application of F); linear density mixing rho_in <- alpha rho_in + (1 - alpha)
 * rho_out (Eq. 14); relative density error (1/N_e) h^3 sum |rho_in - rho_out| (Eq. 15).
 * rsx_scf_create: ctx an FP32 context on a cubic box (kept), V_ext device [N] (kept by
 *   pointer), nocc <= 16, 0 <= alpha < 1.
 * rsx_scf_init: starting orbitals psi0 [nocc][N] (device); Rayleigh-Ritz with T + V_ext;
 *   the first input density is theirs.
 * rsx_scf_step: one SCF iteration with `inner` eigensolver steps; out_host[6] = HF energy
 *   E = 2 sum_i <phi_i, (T + V_ext) phi_i> + 1/2 <rho, V_H> + sum_i <phi_i, Vx phi_i> of
 *   the orbitals entering the iteration, its three parts (one-body, Hartree, exchange),
 *   the relative density error of the previous iteration (0 on the first) and the sum of
 *   the new Ritz values.  Synchronises the stream.
 * Errors: RSX_EINVAL, RSX_ENOMEM, RSX_ECUDA, RSX_ENOTPD (ACE matrix not negative definite). */
typedef struct rsx_scf rsx_scf;
int rsx_scf_create(rsx_scf** scf, rsx_ctx* ctx, const float* V_ext, int nocc, int use_ace, float alpha);
int rsx_scf_init(rsx_scf* scf, const float* psi0, void* stream);
int rsx_scf_step(rsx_scf* scf, int inner, double* out_host, void* stream);
/* What Eq. 14 mixes (before the first rsx_scf_step after rsx_scf_init): 0 the density
 * (default); 1 the states -- the next input orbitals are alpha phi_in + (1 - alpha) P_out
 * phi_in, orthonormalised by the Cholesky factor of their overlap, P_out the projector on
 * the output orbitals' span; the Fock operator then takes V_H and Vx from the input
 * orbitals, and the reported energy is theirs.  Errors: RSX_EINVAL, RSX_ENOMEM. */
int rsx_scf_set_mixing(rsx_scf* scf, int mix_states);
/* Spherical domain for the orbitals (as rsx_eig_set_mask); call before rsx_scf_init. */
int rsx_scf_set_mask(rsx_scf* scf, const float* mask);
int rsx_scf_orbitals(rsx_scf* scf, float* psi_out, void* stream);
const char* rsx_scf_last_error(const rsx_scf* scf);
int rsx_scf_destroy(rsx_scf* scf);

/* Learned preconditioner network: conv3d(2 -> 16) ReLU conv3d(16 -> 16) ReLU conv3d(16 -> 1),
 * 3^3 kernels, zero padding 1, weights used in bf16, FP32 activations; every convolution
 * (forward and data gradient) runs on the tensor cores with each activation split into
 * bf16 hi + lo, FP32 accumulation.
 * Parameters (rsx_net_param_count() floats): w1 [16][2][27], b1 [16], w2 [16][16][27],
 * b2 [16], w3 [1][16][27], b3 [1]; taps t = 9 dz + 3 dy + dx.  Inputs x: device
 * [B][2][D][H][W]; outputs [B][D][H][W].  Loss: mean over voxels at least `border` from
 * every face of (net(x) - target)^2.  rsx_net_loss_grad returns loss and gradients to the
 * host; rsx_net_train_step does one Adam step (beta 0.9 / 0.999, eps 1e-8). */
int rsx_net_create(rsx_net** net, int device);
int rsx_net_param_count(void);
int rsx_net_set_params(rsx_net* net, const float* host_params, int count);
int rsx_net_get_params(rsx_net* net, float* host_params, int count);
int rsx_net_forward(rsx_net* net, const float* x, int B, int D, int H, int W, float* out, void* stream);
int rsx_net_loss_grad(rsx_net* net, const float* x, const float* target, int B, int D, int H, int W, int border,
                      double* loss_host, float* grad_host, void* stream);
int rsx_net_train_step(rsx_net* net, const float* x, const float* target, int B, int D, int H, int W, int border,
                       float lr, double* loss_host, void* stream);
/* Synchronises the stream, then returns (and clears) a deferred device error of the network
 * kernels: RSX_ETIMEOUT when a tensor-core convolution gave up one of its bounded waits
 * (its outputs are then incomplete).  rsx_eig_step checks it after its own synchronisation. */
int rsx_net_sync_status(rsx_net* net, void* stream);
const char* rsx_net_last_error(const rsx_net* net);
int rsx_net_destroy(rsx_net* net);

/* Split-BF16 symmetric contraction on the tensor cores, the K contraction of
 * rsx_casida_K as a standalone building block: C = H H^T + H L^T + L H^T, i.e. S S^T for a
 * panel S = H + L split into bf16 high and low parts (FP32 accumulation, FP64 split-K
 * reduction; C symmetric).  hi, lo: device bf16 [n][ld] row-major, 16-byte aligned,
 * n % 128 == 0, ld % 64 == 0; C: device double [n][n].  Errors: RSX_EINVAL. */
int rsx_syrk_bf16x3(rsx_ctx* ctx, const void* hi, const void* lo, int n, long long ld, double* C, void* stream);

/* Launch profiler (tracing).  While enabled, every kernel the context launches is
 * bracketed by CUDA events recorded on the launching stream; rsx_profile_read waits for
 * the pending events and returns, for kernel id `kernel` (0 <= kernel < rsx_kernel_count()),
 * the summed device time in ms and the number of launches since the last reset.
 * Errors: RSX_EINVAL (null context, kernel out of range). */
int rsx_profile_enable(rsx_ctx* ctx, int on);
int rsx_profile_reset(rsx_ctx* ctx);
int rsx_profile_read(rsx_ctx* ctx, int kernel, double* total_ms, long long* launches);
int rsx_kernel_count(void);
const char* rsx_kernel_name(int kernel);

/* Failure detection, exercised without faulting the GPU (testing aids; the paper has no
 * counterpart).
 * rsx_set_wait_limit: spin rounds a CTA of the context's cooperative kernels (the
 *   grid-wide barrier of the multi-CTA Householder reduction) waits before giving up;
 *   spins < 0 restores the default (2^24 rounds, far beyond any normal wait), 0 makes
 *   every CTA but the last arriver give up at once.  A CTA that gives up marks the
 *   barrier aborted, every CTA leaves at its next barrier, and rsx_sync_status reports
 *   RSX_ETIMEOUT (the call's results are then invalid; the context stays usable).
 * rsx_inject_fault: kind RSX_FAULT_ALLOC makes the workspace allocation after `after`
 *   more successful ones fail with RSX_ENOMEM without touching the device (once);
 *   RSX_FAULT_PIVOT makes the next rsx_ace_build factorise the ACE matrix with its sign
 *   flipped, so that the FP64 Cholesky meets a non-positive pivot and rsx_sync_status
 *   reports RSX_ENOTPD (once); RSX_FAULT_NONE clears both.  Errors: RSX_EINVAL.
 *   The same faults can be armed for every context a process creates through the
 *   environment: RSX_INJECT_FAULT=alloc:N or RSX_INJECT_FAULT=pivot, read at the end of
 *   rsx_create (the count starts after the context's own set-up allocations). */
enum { RSX_FAULT_NONE = 0, RSX_FAULT_ALLOC = 1, RSX_FAULT_PIVOT = 2 };
int rsx_set_wait_limit(rsx_ctx* ctx, long long spins);
int rsx_inject_fault(rsx_ctx* ctx, int kind, int after);

/* Synchronise `stream` and return the first deferred device error since the last call
 * (RSX_ENOTPD, RSX_ETIMEOUT) or a CUDA error; clears the device status word. */
int rsx_sync_status(rsx_ctx* ctx, void* stream);

#ifdef __cplusplus
}
#endif

#endif /* RSX_H */
