// Internal declarations of the sgw library: context, device tables, kernel launchers.
#pragma once

#include <cuda_runtime.h>

#include <complex>
#include <cstdint>
#include <string>
#include <vector>

#include "sgw.h"

namespace sgw {

using cplx = std::complex<double>;

// Status codes written by kernels into the context's device status word.
enum DeviceStatus : int { DEV_OK = 0, DEV_SINGULAR = 1, DEV_TIMEOUT = 2, DEV_BADJOB = 3 };

// One block-diagonal partition of an index range [0, n): for every index v,
// the first index and size of its block and the offset of the block's data
// (row-major n_b x n_b) inside the packed matrix of that wedge point.
struct Partition {
  std::vector<int> sizes;      // per block
  std::vector<int> starts;     // per index: first index of its block
  std::vector<int> isize;      // per index: size of its block
  std::vector<long long> doff; // per index: packed offset of its block
  long long elems = 0;
  // per block: dimension d of its irrep; in a partner-adapted basis the block is d identical
  // m x m copies, m = size / d (0: the block's vectors disagreed on d)
  std::vector<int> dims;
};

// Item of a block-diagonal multiply (see bd_mult).
struct BdItem {
  long long x_off, y_off, m_off;
  int part;
  int pad;
  double2 scale;
};

// Unit of the block-Gram kernel (see gram_*): one <= 32 x 32 tile of one
// output block, one contiguous range of pairs.
struct GramUnit {
  long long a_off, b_off;  // element offsets (pair r0, first tile row) of the A and B operands
  int rows_m, rows_n;      // tile extent
  int r0, r1;              // pair range [r0, r1)
  int slot;                // partial-sum slot (units run largest first; tiles address slots)
  int tri;                 // 1: diagonal tile of a Hermitian block, only elements i <= j
};

// Output tile of a Gram reduction: sums its units (in order) into the packed output.
struct GramTile {
  long long out_off;  // element offset of tile element (0,0) in the output
  int ld;             // row stride of the output block
  int rows_m, rows_n;
  int unit_begin, unit_count;
  int tri;            // 1: only elements i <= j are reduced (the rest is filled by transposition)
};

// Kernel launchers (kernels.cu).
struct BdGeom {
  int U, Vd, Wd;        // Y[u][v][w]
  long long xs_u, xs_v; // strides of X (w contiguous)
  long long ys_u, ys_v;
  int left;             // 1: partition over v (L[v][v']), 0: partition over w (R[w'][w])
  int trans, conj;      // use M^T / conj(M)
  int accumulate;       // Y += ...
  int n_part;           // partition table width (Vd for left, Wd for right)
};
void bd_mult(const BdGeom& g, const double2* X, double2* Y, const double2* M, const BdItem* items, long long nitems,
             const int* p_start, const int* p_size, const long long* p_doff, cudaStream_t st);
void bd_mult(const BdGeom& g, const float2* X, float2* Y, const float2* M, const BdItem* items, long long nitems,
             const int* p_start, const int* p_size, const long long* p_doff, cudaStream_t st);
// chunked variant (hot path): per partition a list of (first output, count <= 8, block start, block size)
void bd_mult2(const BdGeom& g, const double2* X, double2* Y, const double2* M, const BdItem* items, long long nitems,
              const int* nunits, const int4* units, const long long* udoff, int ustride, int max_units,
              cudaStream_t st);
void bd_mult2(const BdGeom& g, const float2* X, float2* Y, const float2* M, const BdItem* items, long long nitems,
              const int* nunits, const int4* units, const long long* udoff, int ustride, int max_units,
              cudaStream_t st);

struct GramGeom {
  long long a_pair, b_pair;  // pair strides
  long long a_row, b_row;    // row strides
  long long k_outer_a, k_outer_b;  // stride of the outer K index
  int k_inner, k_outer;      // K = k_outer * k_inner, inner contiguous
};
void gram_partials(const GramGeom& g, const double2* A, const double2* B, const GramUnit* units, int nunits,
                   double2* partial, cudaStream_t st);
void gram_reduce(const GramTile* tiles, int ntiles, const double2* partial, double2* out, double2 alpha, int accumulate,
                 cudaStream_t st);
void gram_partials(const GramGeom& g, const float2* A, const float2* B, const GramUnit* units, int nunits,
                   float2* partial, cudaStream_t st);
void gram_reduce(const GramTile* tiles, int ntiles, const float2* partial, double2* out, double2 alpha, int accumulate,
                 cudaStream_t st);
void to_c64(const double2* a, float2* b, long long n, cudaStream_t st);
// Hermitian blocks from their upper triangles: out[off + i n + j] = conj(out[off + j n + i]) for
// i > j, and the imaginary part of the diagonal set to zero.
struct HermItem {
  long long off;
  int n, pad;
};
void hermitian_fill(const HermItem* items, int nitems, double2* out, cudaStream_t st);
// Hermitian part of every block: X <- (X + X^dagger) / 2.
void hermitian_part(const HermItem* items, int nitems, double2* X, cudaStream_t st);

// dst = src^dagger per block (conjugate transpose between two blocks of the same size): W at a
// negative bosonic frequency from W at the mirrored positive one.
struct AdjItem {
  long long src_off, dst_off;
  int n, pad;
};
void block_adjoint(const AdjItem* items, int nitems, double2* X, cudaStream_t st);

// tau reflection of P0 in block coordinates: for t in [h, nt) and every item (one auxiliary block
// of a wedge point), P0[t][dst] = M_b P0[nt - 1 - t][src]^T M_b^dagger (M_b n x n at m_off);
// scratch holds (nt - h) packed families.
struct ReflItem {
  long long dst_off, src_off, m_off;
  int n, pad;
};
// the 32 x 32 output tiles of every item (tile row ti, column tj)
struct ReflTile {
  int item, ti, tj, pad;
};
void p0_reflect(const ReflItem* items, const ReflTile* tiles, int ntiles, double2* P0, long long p_elems, int nt, int h,
                const double2* M, double2* scratch, cudaStream_t st);

// out[m][e] = alpha * sum_t T[m][t] in[t * in_ld + e] (+ out if accumulate); T complex (nm x nt).
void series_map(const double2* T, int nm, int nt, const double2* in, long long in_ld, double2* out, long long out_ld,
                long long E, double2 alpha, int accumulate, cudaStream_t st);

// Batched in-place inversion of blocks (Gauss-Jordan, partial pivoting).
struct InvItem {
  long long a_off;   // first source operand (P0(i Omega) block, or Sigma(i w) block)
  long long s_off;   // S block (Dyson) / unused
  long long f_off;   // F = H0 + Sigma_HF block (Dyson) / unused
  long long out_off; // destination block
  int n;
  int m;             // frequency index (Dyson)
  int slot;          // trace partial slot (Dyson number mode)
  double2 weight;    // trace weight (Dyson number mode): partial = (Re weight Tr[G S], -Re weight Tr[G S G S])
};
enum InvMode { INV_W = 0, INV_DYSON_STORE = 1, INV_DYSON_TRACE = 2 };
// A batch of blocks split three ways, each group ordered by n, largest first:
// items [0, nsmall) have n <= 32 (one warp each, largest n small_n); [nsmall, nsmall + nscr)
// n > 90 (one CTA each, global scratch slots of max_n^2); the rest 32 < n <= 90 (one CTA each,
// shared memory, largest n mid_n).  With both side streams set, the groups run concurrently.
struct InvPlan {
  const InvItem* items = nullptr;
  int nitems = 0, nsmall = 0, small_n = 1, nscr = 0, mid_n = 1, max_n = 1;
  cudaStream_t aux[2] = {nullptr, nullptr};
  cudaEvent_t fork = nullptr, join[2] = {nullptr, nullptr};
};
void invert_plan(int mode, const InvPlan& plan, const double2* A, const double2* S, const double2* F, const double* nu,
                 double mu, const double* mu_dev, const double* done_dev, double2* out, double2* trace_partial,
                 double2* scratch, int* status, cudaStream_t st);
void mu_start(double* s, double start_host, const double* start_dev, double lo, double hi, cudaStream_t st);
void mu_update(double* s, const double2* partial, int n, double target, double tol, cudaStream_t st);

// Batched generalised Hermitian eigensolver H C = S C eps (S may be null: identity).
struct EigItem {
  long long h_off, s_off, c_off, e_off;
  int n;
  int pad;
};
void geneig(const EigItem* items, int nitems, int max_n, const double2* H, const double2* S, double2* C, double* eps,
            double2* scratch, cudaStream_t st);

// Deterministic sum of weighted block trace products:
//   result = sum_items w * sum_{a,b in block} X[x_off + a n + b] * Y[y_off + b n + a]
struct TrItem {
  long long x_off, y_off;
  int n;
  int pad;
  double2 w;
};
void trace_products(const TrItem* items, int nitems, const double2* X, const double2* Y, double2* partial,
                    double2* result, cudaStream_t st);
void sum_partials(const double2* partial, int n, double2* result, cudaStream_t st);

void fill_zero(double2* p, long long n, cudaStream_t st);
void axpby(double2* y, const double2* x, long long n, double a, double b, cudaStream_t st);  // y = a y + b x
void max_abs_diff(const double2* a, const double2* b, long long n, unsigned long long* out_bits, cudaStream_t st);
void pack_blocks(const double2* dense, long long dense_ld_mat, int n, const long long* blk_dense_off, const int* blk_n,
                 const long long* blk_pack_off, int nblk, double2* packed, int to_packed, cudaStream_t st);
void g0_closed_form(const double2* C, const double* eps, const long long* row_blk_off, const int* row_blk_n,
                    const long long* row_e_off, long long g_elems, const double* tau, int ntau, double beta, double mu,
                    double2* G, cudaStream_t st);
double mu_bisect_device(const double* eps, const double* wts, int n, double beta, double n_target, double lo, double hi,
                        double* work, cudaStream_t st);

}  // namespace sgw

namespace sgw {
struct TcPlan;  // tensor-core jobs of the chosen form (tc.cu)
// Cached launch tables of one contraction (P0, Sigma or exchange), built once.
struct ContractionPlan {
  bool built = false;
  long long pb = 0, pe = 0;           // pair range [pb, pe) of the orientation's pair list it covers
  int nt_eff = 0;                     // tau values contracted (the first ceil(nt/2) with the P0 reflection)
  int nc = 0;                         // tau values per chunk
  long long items_per_t = 0;          // block-multiply items per tau value
  BdItem *d_A = nullptr, *d_B = nullptr;
  GramUnit* d_units = nullptr;
  GramTile* d_tiles = nullptr;
  std::vector<long long> unit_start, tile_start;  // per tau value (size nt + 1)
  long long max_units_chunk = 0;
  double fl_A_t = 0, fl_B_t = 0, fl_G_t = 0;  // algorithmic flops per tau value of the three stages
};
}  // namespace sgw

// The context.  Host vectors hold the set-up tables; d_* are device copies.
struct sgw_ctx {
  sgw_params p{};
  std::vector<int> mats_f, mats_b;
  int Nk = 0, nao = 0, naux = 0, nt = 0, nwf = 0, nwb = 0;
  int device = -1;  // CUDA device current at sgw_create; the context's memory lives there
  std::string last_error;

  // tau grid and transforms (host, row-major)
  std::vector<double> tau;
  std::vector<sgw::cplx> TF, TFbar, TB, TBbar;  // (nwf x nt), (nt x nwf), (nwb x nt), (nt x nwb)
  std::vector<double> nu_f, nu_b;
  std::vector<double> beta_row;                 // f(beta^-) = beta_row . f(tau)
  std::vector<sgw::cplx> gamma_w;               // gamma = sum_m gamma_w[m] G(i w_m)
  std::vector<double> gl_interp, gl_w;          // values at Gauss-Legendre nodes, weights
  double2 *d_TF = nullptr, *d_TFbar = nullptr, *d_TB = nullptr, *d_TBbar = nullptr;
  double2 *d_beta_row = nullptr, *d_gl_interp = nullptr;
  double* d_nu_f = nullptr;
  double* d_tau = nullptr;

  // symmetry
  bool built = false;
  int nwedge = 0;
  std::vector<int> wedge_k, rep, op, star;
  std::vector<sgw::Partition> part_ao, part_aux;
  std::vector<long long> g_off, p_off;
  long long g_elems = 0, p_elems = 0;
  int max_ao_block = 0, max_aux_block = 0;
  double2 *d_Uao = nullptr, *d_Uaux = nullptr;  // [Nk][n][n]
  std::vector<sgw::cplx> hostU[2];                // host copies, freed after upload
  // partner-adapted bases of the wedge points ([nwedge][n x n] per family), built by
  // build_symmetry only when want_partner is set (host-only query; the GPU path does not use them)
  bool want_partner = false;
  std::vector<std::vector<sgw::cplx>> partner_U[2];
  int *d_ao_start = nullptr, *d_ao_size = nullptr, *d_aux_start = nullptr, *d_aux_size = nullptr;
  long long *d_ao_doff = nullptr, *d_aux_doff = nullptr;
  // chunked unit tables of the orbital (0) and auxiliary (1) partitions, per wedge point
  int* d_nunits[2] = {nullptr, nullptr};
  int4* d_units[2] = {nullptr, nullptr};
  long long* d_udoff[2] = {nullptr, nullptr};
  int ustride[2] = {0, 0};
  int *d_full_start = nullptr, *d_full_size = nullptr;  // one block covering [0, max(nao,naux))
  long long* d_full_doff = nullptr;
  std::vector<int> pair_k1[2], pair_k2[2];

  // inputs in block coordinates
  double2 *d_V[2] = {nullptr, nullptr};  // [npairs][naux][nao][nao]
  float2* d_V32[2] = {nullptr, nullptr};  // complex64 copies for the chosen form (orientation 1 as
                                          // [pair][i][A][a] when the tensor-core chains are used)
  bool use_tc = false;                     // chosen form runs its chains on the tensor cores
  sgw::TcPlan* tc = nullptr;       // whole pair list
  sgw::TcPlan* tc_part = nullptr;  // the last partial pair range asked for
  float2* d_g32 = nullptr;                 // complex64 tau series (chosen form)
  size_t g32_elems = 0;
  double2 *d_H0 = nullptr, *d_S = nullptr;  // packed [g_elems]
  bool have_one_body = false, have_v[2] = {false, false};
  std::vector<long long> v_loaded[2];

  // cached launch tables
  sgw::ContractionPlan plan_p0, plan_sigma, plan_k, plan_rho;
  sgw::ContractionPlan plan_p0_part, plan_sigma_part;  // the last partial pair range asked for
  std::vector<long long> plan_k_wbeg;  // per wedge point: first unit / tile of the exchange plan
  std::vector<long long> plan_k_tbeg;
  // per packed orbital element: block offset, block size, eps offset, row, column, wedge point
  long long *d_el_boff = nullptr, *d_el_eoff = nullptr;
  int *d_el_bn = nullptr, *d_el_i = nullptr, *d_el_j = nullptr, *d_el_w = nullptr;
  // block lists over the wedge: orbital and auxiliary
  std::vector<long long> aob_off, auxb_off;  // packed offset
  std::vector<int> aob_n, auxb_n, aob_w, auxb_w, aob_start, auxb_start;
  // static launch tables of the hot path (built once, so the iteration can be captured in a graph)
  bool tables = false;
  sgw::InvItem *d_w_items = nullptr, *d_dy_items = nullptr;
  int n_w_items = 0, n_dy_items = 0;
  sgw::InvPlan w_plan, dy_plan;   // W solve and Dyson batches (items above, side streams below)
  // W solve over the non-negative bosonic frequencies only (frequency sets closed under
  // n -> -n, sorted): rows [wh_m0, nw_b) are solved, the rest filled as adjoints; wh_m0 < 0: off
  int wh_m0 = -1;
  sgw::InvItem* d_wh_items = nullptr;
  sgw::InvPlan wh_plan;
  sgw::AdjItem* d_wh_adj = nullptr;
  int n_wh_adj = 0;
  cudaStream_t inv_aux[2] = {nullptr, nullptr};
  cudaEvent_t inv_ev[3] = {nullptr, nullptr, nullptr};
  long long* d_hf_tab = nullptr;  // gamma scatter table (dense offsets, packed offsets, sizes, V offsets)
  bool herm = false;  // frequency sets closed under w -> -w: Hermitian blocks are exploited
  // P0^{q_w}(tau) for tau past the middle node from P0^{-q_w}(beta - tau) (set up by
  // sgw_build_irrep_basis when every reflection matrix is block structured)
  bool refl_ok = false;
  sgw::ReflItem* d_refl = nullptr;
  int n_refl = 0;
  sgw::ReflTile* d_refl_tiles = nullptr;
  int n_refl_tiles = 0;
  double2* d_reflM = nullptr;
  sgw::HermItem* d_herm_items[3] = {nullptr, nullptr, nullptr};  // Sigma~(tau), P0(tau), Sigma_HF blocks
  int n_herm_items[3] = {0, 0, 0};
  // iteration buffers and the captured graph
  double2 *d_it_P0 = nullptr, *d_it_P = nullptr, *d_it_S = nullptr, *d_it_H = nullptr;
  double* h_pinned = nullptr;  // host-visible scalars written at the end of a captured iteration
  cudaGraphExec_t it_exec = nullptr;
  cudaGraph_t it_graph = nullptr;
  const void* it_key[4] = {nullptr, nullptr, nullptr, nullptr};
  double it_damping = -1.0;
  long long it_gen = -1, ws_gen = 0;  // workspace generation seen by the captured graph
  int it_warm = 0;
  double2* d_C0 = nullptr;   // eigenvectors of (H0, S) per block (packed)
  double* d_eps0 = nullptr;  // eigenvalues [nwedge][nao]
  double* d_epsw = nullptr;  // weight per eigenvalue (s / N_k * star)
  // workspaces
  double2* d_ws = nullptr;
  size_t ws_bytes = 0;
  int* d_status = nullptr;
  unsigned long long tc_wait_ns = 2000000000ULL;  // limit of each wait in the tensor-core pipeline kernel
  double* d_scalar = nullptr;  // small host-visible results
  double dy_trial_flops = 0.0; // algorithmic flops of one mu-search trial (set by Dyson)
  double prof_trials_seen = 0.0; // trial count (d_scalar[16]) when profiling was last switched on / read
  unsigned long long* d_maxbits = nullptr;

  // launch accounting and optional per-kernel CUDA-event timing
  struct ProfEvent { int id; cudaEvent_t a, b; };
  bool prof_on = false;
  std::vector<std::string> prof_names;
  std::vector<double> prof_ms, prof_flops;
  std::vector<long long> prof_launch;
  std::vector<ProfEvent> prof_pending;
  long long launches = 0;

  sgw_status fail(sgw_status s, const std::string& msg) {
    last_error = msg;
    return s;
  }
};

// Launch through the accounting: kernel class `name`, algorithmic flops, number of kernels; with
// profiling on, CUDA events on the launching stream bracket the launches.
namespace sgw {
template <class F>
inline void run(sgw_ctx* c, const char* name, double flops, int nkern, cudaStream_t st, F&& f) {
  int id = -1;
  for (size_t i = 0; i < c->prof_names.size(); ++i)
    if (c->prof_names[i] == name) { id = (int)i; break; }
  if (id < 0) {
    id = (int)c->prof_names.size();
    c->prof_names.push_back(name);
    c->prof_ms.push_back(0.0);
    c->prof_flops.push_back(0.0);
    c->prof_launch.push_back(0);
  }
  c->prof_flops[id] += flops;
  c->prof_launch[id] += nkern;
  c->launches += nkern;
  if (!c->prof_on) {
    f();
    return;
  }
  cudaEvent_t a, b;
  cudaEventCreate(&a);
  cudaEventCreate(&b);
  cudaEventRecord(a, st);
  f();
  cudaEventRecord(b, st);
  c->prof_pending.push_back({id, a, b});
}

sgw_status lower_from_upper(sgw_ctx* c, int which, double2* X, cudaStream_t st);
size_t workspace_budget();  // bytes the contraction plans may size their intermediates for
// tau values the P0 chains contract for the pair range [pb, pe) (all of them, or the first
// ceil(nt/2) when the whole pair list is asked for and the reflection is set up)
int p0_tau_count(const sgw_ctx* c, long long pb, long long pe);
// P0 for the tau values past p0_tau_count by the reflection (after the chains, which wrote the
// upper triangles of the first ones): mirror, reflect, mirror
sgw_status p0_complete(sgw_ctx* c, double2* P0, int nt_eff, cudaStream_t st);
double gram_elems(const sgw_ctx* c, int nb);  // elements a Gram stage contracts in a block of nb

// tensor-core chains of the chosen form (tc.cu)
bool tc_supported(const sgw_ctx* c);
void tc_free(sgw_ctx* c);
void tc_store_v(const sgw_ctx* c, int which, const double2* V, float2* out, long long npairs, cudaStream_t st);
// Contraction chains over the pairs [pb, pe) of orientation 0 (P0) or 1 (Sigma~): the partial sum
// over those pairs, every output block written (blocks without pairs in the range are zero).
sgw_status tc_polarization(sgw_ctx* c, const double2* G, double2* out, long long pb, long long pe, cudaStream_t st);
sgw_status tc_self_energy(sgw_ctx* c, const double2* G, const double2* P, double2* out, long long pb, long long pe,
                          cudaStream_t st);
}  // namespace sgw

#define CK(call)                                                                               \
  do {                                                                                         \
    cudaError_t e_ = (call);                                                                   \
    if (e_ != cudaSuccess) return c->fail(SGW_ERR_CUDA, std::string(#call) + ": " + cudaGetErrorString(e_)); \
  } while (0)

#define CKS(expr)                      \
  do {                                 \
    sgw_status s_ = (expr);            \
    if (s_ != SGW_OK) return s_;       \
  } while (0)

// set-up helpers (setup.cpp)
namespace sgw {
sgw_status build_grid(sgw_ctx* c);
sgw_status build_symmetry(sgw_ctx* c, const sgw_structure* st);
sgw_status ensure_workspace(sgw_ctx* c, size_t bytes);
sgw_status ensure_g32(sgw_ctx* c, size_t elems);
}  // namespace sgw
