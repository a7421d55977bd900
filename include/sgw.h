/*
 * sgw.h -- C ABI of the symmetry-adapted finite-temperature GW library (sm_103a).
 *
 * The library evaluates one pass of the self-consistent GW method of
 * Dong & Gull, "Symmetry adaptation for self-consistent many-body
 * calculations" (arXiv:2405.09494), restricted to the irreducible wedge of
 * the Brillouin zone and block-diagonalised into the irreducible
 * representations found by simultaneously diagonalising Dirac characters
 * (Sec. 3.4, Algorithm 1):
 *
 *   G(tau) -> P0(tau) [Eq. (P0)] -> P(i Omega) = [I - P0]^{-1} P0 [Eq. (P02P)]
 *          -> Sigma~(tau) [Eq. (sigma)] -> Sigma_HF [Eq. (sigma_hf)]
 *          -> G(i w) = [(i w + mu) S - H0 - Sigma]^{-1} [Eq. (dyson)] -> G(tau).
 *
 * Conventions
 * -----------
 * Complex numbers are interleaved (re, im) doubles ("complex128"); matrices
 * are row-major.  Every tensor argument is a DEVICE pointer owned by the
 * caller unless the comment says "host".  Calls enqueue work on the given
 * CUDA stream and return; results are ready when the stream is.  The
 * library allocates its own device workspaces (on the first call that needs
 * them, reused afterwards) and frees them in sgw_destroy; caller buffers are
 * never freed or kept after a call.  Batched inversions may fork onto two
 * side streams the context owns and join back to the caller's stream with
 * events before the call's next step (also under graph capture).
 *
 * k mesh: Gamma-centred n1 x n2 x n3; point k has fractional coordinates
 * (i1/n1, i2/n2, i3/n3) in the reciprocal basis and flat index
 * (i1*n2 + i2)*n3 + i3.  The wedge (irreducible Brillouin zone) is the list of
 * star representatives returned by sgw_get_wedge, in increasing flat index.
 *
 * Packed block layout ("packed"): after sgw_build_irrep_basis every wedge
 * point w has an orbital partition into blocks I (sizes n_I) and an auxiliary
 * partition into blocks B (sizes n_B) -- one block per irreducible
 * representation of the little group (Sec. 4.3).  A block-diagonal matrix
 * family over the wedge is stored as the concatenation, over w then over
 * blocks, of the n_I x n_I (resp. n_B x n_B) blocks, row-major:
 *   g_elems = sum_w sum_I n_I^2,  p_elems = sum_w sum_B n_B^2.
 * A tau series is [ntau][g_elems] (orbital) or [ntau][p_elems] (auxiliary).
 * Block coordinates of point k are those of the basis U^k = O^{k_w}(a_k) U^{k_w}
 * (rotation of the wedge basis by the operation a_k that carries k_w to k,
 * Eq. (mat_rot)); in that basis every point of a star has the same blocks.
 *
 * Error behaviour: every call returns an sgw_status; SGW_OK means that the
 * work was enqueued (or done, for host-side calls).  Argument errors are
 * detected before anything is enqueued.  Conditions found on the device (a
 * singular or NaN pivot, a tensor-core job that fails its checks, a pipeline
 * wait over its time limit) are recorded in a device status word and returned
 * by the next call that synchronises (sgw_dyson with a chemical-potential
 * search, sgw_iterate, sgw_sync), which clears it; a chemical-potential search
 * that does not converge returns SGW_ERR_NOCONV.  sgw_last_error gives a text
 * for the last failure.
 * A context must be used by one host thread at a time.
 */
#ifndef SGW_H
#define SGW_H

#include <stddef.h>

#ifdef __cplusplus
extern "C" {
#endif

#if defined(__GNUC__)
#define SGW_API __attribute__((visibility("default")))
#else
#define SGW_API
#endif

typedef struct sgw_ctx sgw_ctx;
typedef struct CUstream_st* sgw_stream; /* a cudaStream_t; NULL is the legacy default stream */

typedef enum {
  SGW_OK = 0,
  SGW_ERR_ARG = 1,           /* invalid argument or size                                  */
  SGW_ERR_CUDA = 2,          /* a CUDA runtime call failed                                 */
  SGW_ERR_OOM = 3,           /* device allocation failed                                   */
  SGW_ERR_SINGULAR = 4,      /* zero pivot in a W solve or Dyson inversion                 */
  SGW_ERR_NOCONV = 5,        /* chemical-potential bisection did not bracket / converge    */
  SGW_ERR_TIMEOUT = 6,       /* a bounded device wait ran out (sgw_set_wait_limit)         */
  SGW_ERR_UNIMPLEMENTED = 7, /* feature not built                                          */
  SGW_ERR_STATE = 8          /* call out of order (e.g. before sgw_build_irrep_basis)       */
} sgw_status;

typedef enum {
  SGW_FP64 = 0,       /* plain form: complex128 everywhere                                  */
  SGW_MIXED_FP32 = 1  /* chosen form: V-G-V and V-G-P-V chains in FP32, rest FP64            */
} sgw_precision;

/* Problem parameters.  The Matsubara index lists are host arrays copied at
 * sgw_create: fermionic frequencies w_n = (2n+1) pi / beta, bosonic
 * Omega_n = 2 n pi / beta (Sec. 4.1 and Eq. (P02P)).  Imaginary time is
 * represented on the ntau Chebyshev roots tau_j = beta (1 - cos(pi (j+1/2)/ntau)) / 2. */
typedef struct {
  int nk[3];
  int nao;          /* orbitals per cell                                          */
  int naux;         /* auxiliary (density-fitting) functions per cell             */
  int ntau;         /* Chebyshev nodes on [0, beta]                               */
  int nw_f;         /* number of fermionic Matsubara indices (>= ntau)            */
  int nw_b;         /* number of bosonic Matsubara indices (>= ntau)              */
  const int* mats_f; /* host [nw_f]                                               */
  const int* mats_b; /* host [nw_b]                                               */
  double beta;      /* inverse temperature (1/Ha)                                 */
  double n_elec;    /* electrons per cell, both spins (Sec. 4.1)                  */
  int spin_factor;  /* 2 for the spin-restricted closed shell                     */
  int loop_sign;    /* +1 physical sign of the bare bubble (default), -1 literal  */
  int precision;    /* sgw_precision                                              */
} sgw_params;

/* Crystal description for the symmetry analysis (Sec. 3, Algorithm 1).
 * lattice: row-major 3x3 whose COLUMNS are the primitive vectors (Cartesian).
 * An operation {R|v} maps r to R r + v (Cartesian, R orthogonal).  Every atom
 * carries the same shell list; a shell of angular momentum l holds the 2l+1
 * real spherical harmonics m = -l..l (Y_l0 = Y_l^0, Y_{l,m>0} = sqrt2 (-1)^m
 * Re Y_l^m, Y_{l,m<0} = sqrt2 (-1)^m Im Y_l^|m|, Condon-Shortley Y_l^m).  The
 * basis order is atom, shell, m.  A structure with one operation (the
 * identity) means "no symmetry": the wedge is the whole mesh and every
 * matrix is one block. */
typedef struct {
  double lattice[9];
  int natom;
  const double* positions;    /* host [natom][3]                                */
  int nops;
  const double* rotations;    /* host [nops][3][3] row-major                    */
  const double* translations; /* host [nops][3]                                 */
  int n_ao_shells;
  const int* ao_shells;       /* host [n_ao_shells] angular momenta             */
  int n_aux_shells;
  const int* aux_shells;      /* host [n_aux_shells]                            */
} sgw_structure;

typedef struct {
  int nkpts;            /* N_k                                                  */
  int nwedge;           /* wedge points                                         */
  long long g_elems;    /* packed orbital elements (per tau or frequency)        */
  long long p_elems;    /* packed auxiliary elements                             */
  long long npairs;     /* momentum pairs per V orientation = nwedge * nkpts     */
  int max_ao_block;
  int max_aux_block;
} sgw_layout;

typedef struct {
  int iterations;
  double mu;
  double n_elec;        /* particle number reached                              */
  double max_dsigma;    /* max |Sigma_new - Sigma_old| of the last iteration    */
  double energy[4];     /* E, E_one_body, E_hf, E_c (real parts)                 */
  double energy_imag;   /* Im E                                                  */
} sgw_iter_stats;

/* ---- context -------------------------------------------------------------- */

/* Create a context on the current CUDA device.  Builds the tau grid and the
 * Matsubara transform matrices (Sec. 4.1; least-squares inverse of the
 * forward map) on the host.  Returns SGW_ERR_ARG for inconsistent sizes. */
SGW_API sgw_status sgw_create(const sgw_params* params, sgw_ctx** out);
/* Free every library-owned resource (device workspaces, tables). */
SGW_API sgw_status sgw_destroy(sgw_ctx* ctx);
/* Static text for a status code. */
SGW_API const char* sgw_status_str(sgw_status s);
/* Copy the detail text of the last failure of this context into buf (host). */
SGW_API sgw_status sgw_last_error(const sgw_ctx* ctx, char* buf, size_t len);
/* Wait for the stream, then return the device status word (singular pivot...). */
SGW_API sgw_status sgw_sync(sgw_ctx* ctx, sgw_stream stream);

/* ---- a1: irrep basis (set-up, once) ---------------------------------------- */

/* Algorithm 1: orbital representations O^k(a) (Eq. (basis_rot)), projective
 * representations and factor systems (Eqs. (projrep), (factor)), Dirac
 * characters of the little groups (Eq. (dirac)), simultaneous
 * diagonalisation into U^k (Sec. 3.4), stars and the wedge (Sec. 4.2), for
 * the orbital and the auxiliary basis.  Host analysis plus a batched FP64
 * Jacobi eigensolver on the device; synchronous.  Fills *out. */
SGW_API sgw_status sgw_build_irrep_basis(sgw_ctx* ctx, const sgw_structure* st, sgw_layout* out);
/* Host outputs: wedge_k[nwedge] flat indices of the wedge points; rep[nkpts]
 * wedge index of the star of each k; op[nkpts] index of the operation a_k
 * with a_k k_w = k (mod K).  Any pointer may be NULL. */
SGW_API sgw_status sgw_get_wedge(const sgw_ctx* ctx, int* wedge_k, int* rep, int* op);
/* Host output: sizes of the blocks of wedge point w; which = 0 orbital,
 * 1 auxiliary.  *nblocks receives the count; sizes needs room for nao
 * (resp. naux) entries. */
SGW_API sgw_status sgw_get_blocks(const sgw_ctx* ctx, int which, int w, int* nblocks, int* sizes);
/* Host output: the momentum pairs (k1[p], k2[p]) of orientation `which`:
 * 0 = polarization pairs (k, k + q_w) ordered [w][k]; 1 = self-energy pairs
 * (k_w, k2) ordered [w][k2] (Sec. 5.2: one momentum in the wedge, the other
 * anywhere in the zone). */
SGW_API sgw_status sgw_get_pairs(const sgw_ctx* ctx, int which, int* k1, int* k2);
/* Device output [nkpts][n][n]: the basis U^k (n = nao or naux, which = 0/1). */
SGW_API sgw_status sgw_get_basis(const sgw_ctx* ctx, int which, void* U, sgw_stream stream);

/* ---- inputs ------------------------------------------------------------------ */

/* H0^k and S^k for every k of the mesh, [nkpts][nao][nao] complex128 in the
 * orbital (AO) basis; the wedge blocks U^dagger X U are kept (Eq. (mat_blk)). */
SGW_API sgw_status sgw_load_one_body(sgw_ctx* ctx, const void* H0, const void* S, sgw_stream stream);
/* V^{k1,k2}_{Q,ij} for pairs [first, first + count) of orientation `which`,
 * [count][naux][nao][nao] complex128 in the AO basis (V^{k,k'}_{Q,ij} =
 * conj(V^{k',k}_{Q,ji})).  Transformed to block coordinates (Eq. (C_blk) with
 * an orthonormal auxiliary basis) and kept on the device: orientation 0 with
 * its auxiliary index in the basis U^{q} (q = k2 - k1), orientation 1 in the
 * basis conj(U^{k1 - k2}) -- the basis in which Eq. (sigma) meets P^q without
 * a further rotation.  The input buffer may be reused after the stream
 * reaches this call. */
SGW_API sgw_status sgw_load_v(sgw_ctx* ctx, int which, long long first, long long count, const void* V,
                              sgw_stream stream);

/* ---- hot path -------------------------------------------------------------- */

/* Non-interacting start: mu0 by bisection on the Fermi sum of the eigenvalues
 * of (H0, S) (Sec. 4.1 particle number) and G0(tau) in closed form (Eq. (dyson)
 * with Sigma = 0).  Synchronous for mu (*mu_out is host).  G_tau: packed
 * [ntau][g_elems]. */
SGW_API sgw_status sgw_g0(sgw_ctx* ctx, double* mu_out, void* G_tau, sgw_stream stream);
/* a2 + a3: P0^q(tau) for every wedge q from G(tau) (Eq. (P0), Algorithm 3):
 * G of every point of the zone is read through the star map (no unfolding),
 * X_Q = G^k(-tau) V_Q G^{k+q}(tau), P0 += X V^dagger over the diagonal
 * auxiliary blocks.  G_tau packed [ntau][g_elems]; P0_tau packed [ntau][p_elems].
 * Each block of P0 is Hermitian when G^k(tau) is Hermitian and the two loaded
 * orientations of V satisfy V^{k2,k1}_Q = (V^{k1,k2}_Q)^dagger.  When both
 * Matsubara sets given to sgw_create are closed under w -> -w (fermionic n ->
 * -n-1, bosonic n -> -n; the transforms then keep Hermiticity exactly), only
 * the tiles on and above the diagonal are contracted and the strict lower
 * triangle is written as the conjugate transpose of the upper one (here and in
 * sgw_self_energy); otherwise every tile is contracted. */
SGW_API sgw_status sgw_polarization(sgw_ctx* ctx, const void* G_tau, void* P0_tau, sgw_stream stream);
/* a3 restricted to the momentum pairs [pair_begin, pair_end) of the
 * polarization pair list (orientation 0 of sgw_get_pairs, ordered
 * p = w N_k + k for the pair (k, k + q_w)): the partial sum of Eq. (P0) over
 * those pairs, with the same normalisation (s / N_k).  The sum of the partial
 * results of ranges that cover the list once equals sgw_polarization (the
 * pair units of Algorithm 3 are independent, Sec. 5.2): one rank per range,
 * then one sum over the ranks.  Every block of P0_tau is written (blocks of
 * wedge points with no pair in the range are zero).  0 <= pair_begin <=
 * pair_end <= nwedge N_k, else SGW_ERR_ARG; an empty range gives zeros.  The
 * context keeps the plan of the last partial range asked for (and that of
 * the whole list); asking for another range rebuilds it. */
SGW_API sgw_status sgw_polarization_pairs(sgw_ctx* ctx, const void* G_tau, void* P0_tau, long long pair_begin,
                                          long long pair_end, sgw_stream stream);
/* a4 + a5 + a6: P0(tau) -> P0(i Omega) -> P = [I - P0]^{-1} P0 per block
 * (Eq. (P02P), FP64 in both forms) -> P(tau). */
SGW_API sgw_status sgw_screened_interaction(sgw_ctx* ctx, const void* P0_tau, void* P_tau, sgw_stream stream);
/* a7: Sigma~^k(tau) for every wedge k (Eq. (sigma), Algorithm 4), diagonal
 * orbital blocks only.  Sigma_tau packed [ntau][g_elems]. */
SGW_API sgw_status sgw_self_energy(sgw_ctx* ctx, const void* G_tau, const void* P_tau, void* Sigma_tau,
                                   sgw_stream stream);
/* a7 restricted to the momentum pairs [pair_begin, pair_end) of the
 * self-energy pair list (orientation 1, p = w N_k + k2 for the pair (k_w, k2)):
 * the partial sum of Eq. (sigma) over those pairs (Algorithm 4's pair units),
 * normalisation -1/N_k; the partial results of ranges that cover the list once
 * add up to sgw_self_energy.  Ranges, zero blocks and errors as in
 * sgw_polarization_pairs. */
SGW_API sgw_status sgw_self_energy_pairs(sgw_ctx* ctx, const void* G_tau, const void* P_tau, void* Sigma_tau,
                                         long long pair_begin, long long pair_end, sgw_stream stream);
/* The paper has no counterpart to this entry point: it is sgw_screened_interaction for
 * callers that may not allocate device memory when they call (code running while a CUDA graph
 * is being captured, where cudaMalloc is not permitted, or applications that fix their device
 * memory at start-up).  Same inputs, outputs and result; its scratch (the P0 and P
 * frequency series) lives in a fixed 64 MiB array inside the library image instead of the
 * context workspace, so every GPU that loads the library holds those 64 MiB until the process
 * exits.  It allocates nothing: no cudaMalloc, cudaFree or allocating library routine.
 * Limits: 2 * nw_b * p_elems <= 4 Mi complex numbers and auxiliary blocks of at most 90;
 * larger problems get SGW_ERR_ARG with a message (use sgw_screened_interaction).  The
 * context must have run sgw_screened_interaction once (set-up that allocates the launch
 * tables this call reuses), else SGW_ERR_STATE; SGW_ERR_STATE too when the current device is
 * not the one that was current at sgw_create.  A refused call writes nothing.  With
 * sgw_profile_enable on, its kernels are counted as those of sgw_screened_interaction ("ft",
 * "w_solve").  The first call on a device looks up the
 * array's device address (cudaGetSymbolAddress, with that device current); make that first
 * call before any stream capture.  All calls share the array: calls that overlap on the GPU
 * (on different streams, or from different contexts) race and must be serialised by the
 * caller.  Nothing in the array needs to start at zero (both series are overwritten). */
SGW_API sgw_status sgw_screened_interaction_noalloc(sgw_ctx* ctx, const void* P0_tau, void* P_tau,
                                                    sgw_stream stream);
/* a11: Sigma_HF = J + K from gamma = -G(beta^-) (Eq. (sigma_hf)); packed [g_elems]. */
SGW_API sgw_status sgw_hartree_fock(sgw_ctx* ctx, const void* G_tau, void* Sigma_hf, sgw_stream stream);
/* a8 + a9 + a10: Sigma~(tau) -> Sigma~(i w); G(i w) = [(i w + mu) S - H0 -
 * Sigma_HF - Sigma~(i w)]^{-1} per block (Eq. (dyson)); G(tau).  With
 * search_mu != 0, mu solves N(mu) = (s/N_k) sum_k Tr[gamma^k S^k] = n_elec
 * by Newton's method kept inside the bracket [-20, 20] (N'(mu) from
 * dG/dmu = -G S G; a Newton point outside the current bracket, or one that
 * follows a trial which did not halve |N - n_elec|, is replaced by the
 * bracket's midpoint), starting from *mu_inout (the midpoint when outside
 * the bracket); it stops at |N - n_elec| <= 1e-11 or after 64 trials, and is
 * synchronous in that case.  *mu_inout is host: the start (or the fixed mu
 * without the search) in, the result out.  A search that ends without meeting
 * the tolerance (n_elec out of reach in [-20, 20]) returns SGW_ERR_NOCONV with
 * *mu_inout and G_tau at its last trial. */
SGW_API sgw_status sgw_dyson(sgw_ctx* ctx, const void* Sigma_tau, const void* Sigma_hf, double* mu_inout,
                             int search_mu, void* G_tau, sgw_stream stream);
/* a12: total energy (Galitskii-Migdal form; the paper defines none) into
 * host e_out[5] = {Re E, Re E_1, Re E_HF, Re E_c, Im E}.  Synchronous. */
SGW_API sgw_status sgw_energy(sgw_ctx* ctx, const void* G_tau, const void* Sigma_hf, const void* Sigma_tau,
                              double* e_out, sgw_stream stream);
/* a2..a12 repeated: P0 -> P -> Sigma~, Sigma_HF -> damping
 * Sigma <- (1-damping) Sigma_old + damping Sigma_new -> Dyson with mu search,
 * until max |Sigma_new - Sigma_old| < tol or max_iter passes.  G_tau
 * (in/out), Sigma_tau, Sigma_hf (in/out; zero on the first pass) are packed;
 * *mu is host in/out: each pass's mu search (as in sgw_dyson) starts from the
 * mu of the pass before, the first from *mu.  Synchronous; fills *stats
 * (host, may be NULL).  A pass whose mu search does not converge stops the
 * loop with SGW_ERR_NOCONV. */
SGW_API sgw_status sgw_iterate(sgw_ctx* ctx, int max_iter, double damping, double tol, void* G_tau,
                               void* Sigma_tau, void* Sigma_hf, double* mu, sgw_iter_stats* stats,
                               sgw_stream stream);

/* ---- unfolding -------------------------------------------------------------- */

/* a2 made explicit: packed series [nt][elems] -> AO family over the whole zone
 * [nkpts][nt][n][n], X^k = U^k X_block^{w(k)} U^k^dagger (Eqs. (mat_rot),
 * (mat_blk)).  which = 0 orbital (g_elems), 1 auxiliary (p_elems). */
SGW_API sgw_status sgw_unfold(sgw_ctx* ctx, int which, int nt, const void* packed, void* ao_full,
                              sgw_stream stream);

/* ---- host-only set-up queries (no device is touched) ----------------------- */

/* The tau nodes and transform matrices that sgw_create builds (Sec. 4.1,
 * Eq. (P02P)): tau[ntau]; TF [nw_f][ntau], TFbar [ntau][nw_f], TB [nw_b][ntau],
 * TBbar [ntau][nw_b] as interleaved complex (host).  Any pointer may be NULL. */
SGW_API sgw_status sgw_host_grid(const sgw_params* params, double* tau, double* TF, double* TFbar, double* TB,
                                 double* TBbar);
/* The space-group analysis of sgw_build_irrep_basis (Algorithm 1, Secs. 3-4.2)
 * without the device: *nwedge, rep[nkpts] (wedge index of each k), and the
 * block sizes of every wedge point as zero-terminated rows
 * ao_blocks[nwedge][nao + 1], aux_blocks[nwedge][naux + 1] (host; rows need
 * room for nkpts wedge points).  Any output but nwedge may be NULL. */
SGW_API sgw_status sgw_host_symmetry(const sgw_params* params, const sgw_structure* st, int* nwedge, int* rep,
                                     int* ao_blocks, int* aux_blocks);
/* Irrep dimension d of every block of sgw_host_symmetry, in the same zero-terminated row layout
 * (ao_dims[nwedge][nao + 1], aux_dims[nwedge][naux + 1], host; rows need room for nkpts wedge
 * points): in a partner-adapted basis a block of size s is d identical (s / d) x (s / d) copies
 * (Sec. 3.4, the irreducible decomposition of the orbital representation).  d comes from the
 * block's Dirac-character eigenvalues lambda_c (Eq. (dirac)): d^2 = h / sum_c |lambda_c|^2 / n_c
 * over the classes c of the little co-group of order h.  A 0 marks a block whose vectors
 * disagreed on d.  Any output but nwedge may be NULL. */
SGW_API sgw_status sgw_host_irrep_dims(const sgw_params* params, const sgw_structure* st, int* nwedge, int* ao_dims,
                                       int* aux_dims);
/* Partner-adapted bases of one family (family 0: orbitals, 1: auxiliary) at every wedge point:
 * U[nwedge][n][n] interleaved complex (host, room for nkpts wedge points), column j a basis vector
 * in the AO basis.  The blocks are those of sgw_host_symmetry, in the same order.  Within a block
 * of irrep dimension d and size s = m d, column i m + a is partner i of copy a, so every
 * operator that commutes with the little group's projective representation is I_d (x) A there
 * (Sec. 3.4, Schur's lemma).  Blocks with d = 1 keep the basis of sgw_build_irrep_basis.  Not
 * used by the device path. */
SGW_API sgw_status sgw_host_partner_basis(const sgw_params* params, const sgw_structure* st, int family, int* nwedge,
                                          double* U);

/* ---- instrumentation (not part of the method) ---------------------------- */

/* Time limit (ns) of each wait inside the chosen form's tensor-core pipeline
 * kernel (a stage of copies landing, a stage split, an accumulator filled or
 * drained), applied from the next launch on; 2 s when the context is created.
 * A wait over the limit stops the kernel's CTA cleanly (its copies in flight
 * are waited for, its tensor memory freed) and records SGW_ERR_TIMEOUT, which
 * the next synchronising call returns; results of that call are then invalid,
 * the context stays usable.  0 gives up at the first wait that is not
 * already satisfied (for tests of this path).  Not part of the method. */
SGW_API sgw_status sgw_set_wait_limit(sgw_ctx* ctx, unsigned long long ns);

/* Turn per-kernel CUDA-event timing on (1) or off (0).  Events are recorded on
 * the stream each kernel is launched on.  Launch counts and algorithmic flop
 * counts are always kept. */
SGW_API sgw_status sgw_profile_enable(sgw_ctx* ctx, int on);
/* Synchronise the pending events and report, per kernel class, the summed
 * device time (ms), the algorithmic flops (8 per complex multiply-add of the
 * block-sparse method, counted once) and the launch count since the last
 * reset.  names: host [max_entries][48] chars; ms, gflop: host [max_entries];
 * launches: host [max_entries]; *n_out receives the number of classes. */
SGW_API sgw_status sgw_profile_read(sgw_ctx* ctx, int max_entries, char* names, double* ms, double* gflop,
                                    long long* launches, int* n_out, int reset);

#ifdef __cplusplus
}
#endif
#endif /* SGW_H */
