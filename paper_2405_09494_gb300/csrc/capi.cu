// C ABI of the sgw library: context, loaders and the symmetry-adapted GW steps.
#include <algorithm>
#include <cmath>
#include <cstdlib>
#include <cstring>
#include <string>
#include <type_traits>

#include "sgw_internal.h"

using namespace sgw;

namespace {

template <typename T>
sgw_status upload(sgw_ctx* c, T*& d, const std::vector<T>& h) {
  if (d) cudaFree(d);
  d = nullptr;
  if (h.empty()) return SGW_OK;
  if (cudaMalloc(reinterpret_cast<void**>(&d), h.size() * sizeof(T)) != cudaSuccess)
    return c->fail(SGW_ERR_OOM, "device table allocation failed");
  if (cudaMemcpy(d, h.data(), h.size() * sizeof(T), cudaMemcpyHostToDevice) != cudaSuccess)
    return c->fail(SGW_ERR_CUDA, "device table upload failed");
  return SGW_OK;
}

template <typename T>
void dfree(T*& p) {
  if (p) cudaFree(p);
  p = nullptr;
}

inline cudaStream_t S(sgw_stream s) { return reinterpret_cast<cudaStream_t>(s); }


double2 z(double re, double im = 0.0) { return make_double2(re, im); }

void free_plan(ContractionPlan& p) {
  dfree(p.d_A);
  dfree(p.d_B);
  dfree(p.d_units);
  dfree(p.d_tiles);
  p = ContractionPlan();
}

}  // namespace

// Device memory the contraction plans may size their intermediates for: SGW_WORKSPACE_GB when set,
// otherwise 64 GiB or half of the device memory free when the plan is built, whichever is less (the
// tau chunk of the chains grows with it: V is then read from memory once per chunk).
size_t sgw::workspace_budget() {
  const char* e = std::getenv("SGW_WORKSPACE_GB");
  double gb = 64.0;
  if (e) {
    gb = std::atof(e);
  } else {
    size_t free_b = 0, total_b = 0;
    if (cudaMemGetInfo(&free_b, &total_b) == cudaSuccess) gb = std::min(gb, 0.5 * (double)free_b / (1ull << 30));
  }
  if (gb < 0.5) gb = 0.5;
  return (size_t)(gb * (1ull << 30));
}

namespace sgw {
// single-precision copies of the tau series used by the chosen form (kept apart from the workspace)
sgw_status ensure_g32(sgw_ctx* c, size_t elems) {
  if (elems <= c->g32_elems) return SGW_OK;
  if (c->d_g32) cudaFree(c->d_g32);
  c->d_g32 = nullptr;
  c->g32_elems = 0;
  if (cudaMalloc(&c->d_g32, elems * sizeof(float2)) != cudaSuccess) return c->fail(SGW_ERR_OOM, "complex64 buffers");
  c->g32_elems = elems;
  ++c->ws_gen;  // a captured iteration that used the old buffer must be re-captured
  return SGW_OK;
}
sgw_status ensure_workspace(sgw_ctx* c, size_t bytes) {
  if (bytes <= c->ws_bytes) return SGW_OK;
  // fault injection on the host: SGW_FAIL_ALLOC_ABOVE_MB makes any larger workspace request fail
  // as an allocation failure would (the context keeps its current workspace and stays usable)
  if (const char* lim = std::getenv("SGW_FAIL_ALLOC_ABOVE_MB"))
    if ((double)bytes > std::atof(lim) * (1 << 20))
      return c->fail(SGW_ERR_OOM, "workspace allocation failed (injected by SGW_FAIL_ALLOC_ABOVE_MB)");
  if (c->d_ws) cudaFree(c->d_ws);
  c->d_ws = nullptr;
  c->ws_bytes = 0;
  if (cudaMalloc(&c->d_ws, bytes) != cudaSuccess) return c->fail(SGW_ERR_OOM, "workspace allocation failed");
  c->ws_bytes = bytes;
  ++c->ws_gen;
  return SGW_OK;
}
}  // namespace sgw

// ---------------------------------------------------------------------------
// small kernels of the Hartree term and embeddings
// ---------------------------------------------------------------------------
__global__ void k_hartree(const double2* __restrict__ V, const double2* __restrict__ rho, const int* __restrict__ el_i,
                          const int* __restrict__ el_j, const int* __restrict__ el_w, const long long* __restrict__ vw,
                          long long g_elems, int naux, int nao, double scale, double2* __restrict__ out) {
  for (long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x; e < g_elems;
       e += (long long)gridDim.x * blockDim.x) {
    const double2* Vp = V + vw[el_w[e]] + (long long)el_i[e] * nao + el_j[e];
    double sx = 0, sy = 0;
    const long long st = (long long)nao * nao;
    for (int A = 0; A < naux; ++A) {
      const double2 v = Vp[A * st], r = rho[A];
      sx += v.x * r.x - v.y * r.y;
      sy += v.x * r.y + v.y * r.x;
    }
    out[e] = make_double2(scale * sx, scale * sy);
  }
}

// ---------------------------------------------------------------------------
// helpers on the context
// ---------------------------------------------------------------------------
static sgw_status need_built(sgw_ctx* c) {
  if (!c) return SGW_ERR_ARG;
  if (!c->built) return c->fail(SGW_ERR_STATE, "sgw_build_irrep_basis has not been called");
  return SGW_OK;
}

static long long vsize(const sgw_ctx* c) { return (long long)c->naux * c->nao * c->nao; }

// Block multiply over the orbital (kind 0) or auxiliary (kind 1) partitions.  FP64 is bound by
// the FP64 pipe and runs one output per thread (fewest registers, no predicated slots); FP32
// uses the chunked variant where it reuses operands (right multiplies, large auxiliary blocks).
static void bdm(sgw_ctx* c, int kind, const BdGeom& g, const double2* X, double2* Y, const double2* M,
                const BdItem* items, long long nitems, cudaStream_t st) {
  if (kind == 0)
    bd_mult(g, X, Y, M, items, nitems, c->d_ao_start, c->d_ao_size, c->d_ao_doff, st);
  else
    bd_mult(g, X, Y, M, items, nitems, c->d_aux_start, c->d_aux_size, c->d_aux_doff, st);
}
static void bdm(sgw_ctx* c, int kind, const BdGeom& g, const float2* X, float2* Y, const float2* M,
                const BdItem* items, long long nitems, cudaStream_t st) {
  if (kind == 0 && g.left)
    bd_mult(g, X, Y, M, items, nitems, c->d_ao_start, c->d_ao_size, c->d_ao_doff, st);
  else
    bd_mult2(g, X, Y, M, items, nitems, c->d_nunits[kind], c->d_units[kind], c->d_udoff[kind], c->ustride[kind],
             c->ustride[kind], st);
}

// Build the block-diagonal multiply geometry for a [U][Vd][Wd] contiguous tensor.
static BdGeom geom(int U, int Vd, int Wd, int left, int trans, int conj, int accumulate, int n_part) {
  BdGeom g;
  g.U = U;
  g.Vd = Vd;
  g.Wd = Wd;
  g.xs_v = Wd;
  g.xs_u = (long long)Vd * Wd;
  g.ys_v = Wd;
  g.ys_u = (long long)Vd * Wd;
  g.left = left;
  g.trans = trans;
  g.conj = conj;
  g.accumulate = accumulate;
  g.n_part = n_part;
  return g;
}

// Gram units/tiles for one output block family.  out block of size nb at out_off (ld nb);
// A rows start at a_off (+ row * a_row), B rows at b_off; pairs [0, npair) with strides.
// With herm, the output block is Hermitian: tiles strictly below the diagonal are left out (the
// caller fills them by conjugate transposition).
static void add_gram_block(std::vector<GramUnit>& units, std::vector<GramTile>& tiles, long long unit_base, int nb,
                           long long out_off, long long a_off, long long b_off, long long a_row, long long b_row,
                           int npair, long long kwork, long long target = (1LL << 20), bool herm = false) {
  // balanced square tiles of at most 32 rows; in a Hermitian block the diagonal tiles contract
  // only their elements on and above the diagonal
  const int nt_side = (nb + 31) / 32;
  const int ts = (nb + nt_side - 1) / nt_side;
  for (int tm = 0; tm < nb; tm += ts)
    for (int tn = herm ? tm : 0; tn < nb; tn += ts) {
      const int rm = std::min(ts, nb - tm), rn = std::min(ts, nb - tn);
      long long per_pair = (long long)rm * rn * kwork / (herm && tm == tn ? 2 : 1);
      long long chunk = std::max(1LL, target / std::max(1LL, per_pair));
      if (chunk > npair) chunk = npair;
      // spread the pairs evenly over the units of this tile
      const long long nun = (npair + chunk - 1) / chunk;
      chunk = (npair + nun - 1) / nun;
      const int tri = herm && tm == tn ? 1 : 0;
      GramTile t;
      t.out_off = out_off + (long long)tm * nb + tn;
      t.ld = nb;
      t.rows_m = rm;
      t.rows_n = rn;
      t.tri = tri;
      t.unit_begin = (int)((long long)units.size() - unit_base);
      int cnt = 0;
      for (long long r0 = 0; r0 < npair; r0 += chunk) {
        GramUnit u;
        u.rows_m = rm;
        u.rows_n = rn;
        u.r0 = (int)r0;
        u.r1 = (int)std::min<long long>(npair, r0 + chunk);
        u.a_off = a_off + (long long)tm * a_row;
        u.b_off = b_off + (long long)tn * b_row;
        u.slot = (int)((long long)units.size() - unit_base);
        u.tri = tri;
        units.push_back(u);
        ++cnt;
      }
      t.unit_count = cnt;
      tiles.push_back(t);
    }
}

// Gram units carry the pair offset of their first pair: shift a_off / b_off by r0 pairs.
static void finalize_units(std::vector<GramUnit>& units, size_t from, long long a_pair, long long b_pair) {
  for (size_t i = from; i < units.size(); ++i) {
    units[i].a_off += (long long)units[i].r0 * a_pair;
    units[i].b_off += (long long)units[i].r0 * b_pair;
  }
}

// Order the units of one launch [from, end) largest first (their slots keep the tiles' addressing).
static void schedule_units(std::vector<GramUnit>& units, size_t from, long long kwork) {
  std::stable_sort(units.begin() + from, units.end(), [&](const GramUnit& a, const GramUnit& b) {
    return (long long)a.rows_m * a.rows_n * (a.r1 - a.r0) > (long long)b.rows_m * b.rows_n * (b.r1 - b.r0);
  });
  (void)kwork;
}

// Target multiply-adds per unit so that a launch of `work` fills the GPU several times over:
// about 32 units per SM, i.e. six or more waves of the five resident CTAs per SM, so the last
// wave's idle SMs cost little (at 8 units per SM the Gram stages ran two waves and the SMs were
// busy 81% of the time).
static long long unit_target(double work) {
  const double t = work / (152.0 * 32.0);
  return std::max(1LL << 14, std::min(1LL << 22, (long long)t));
}

// ---------------------------------------------------------------------------
// context
// ---------------------------------------------------------------------------
extern "C" SGW_API const char* sgw_status_str(sgw_status s) {
  switch (s) {
    case SGW_OK: return "ok";
    case SGW_ERR_ARG: return "invalid argument";
    case SGW_ERR_CUDA: return "CUDA error";
    case SGW_ERR_OOM: return "out of device memory";
    case SGW_ERR_SINGULAR: return "singular matrix";
    case SGW_ERR_NOCONV: return "no convergence";
    case SGW_ERR_TIMEOUT: return "device wait timed out";
    case SGW_ERR_UNIMPLEMENTED: return "not implemented";
    case SGW_ERR_STATE: return "call out of order";
  }
  return "unknown status";
}

extern "C" SGW_API sgw_status sgw_last_error(const sgw_ctx* ctx, char* buf, size_t len) {
  if (!ctx || !buf || len == 0) return SGW_ERR_ARG;
  std::strncpy(buf, ctx->last_error.c_str(), len - 1);
  buf[len - 1] = 0;
  return SGW_OK;
}

extern "C" SGW_API sgw_status sgw_create(const sgw_params* p, sgw_ctx** out) {
  if (!p || !out) return SGW_ERR_ARG;
  *out = nullptr;
  if (p->nk[0] < 1 || p->nk[1] < 1 || p->nk[2] < 1 || p->nao < 1 || p->naux < 1 || p->ntau < 2 ||
      p->nw_f < p->ntau || p->nw_b < p->ntau || !p->mats_f || !p->mats_b || !(p->beta > 0) ||
      (p->loop_sign != 1 && p->loop_sign != -1) || p->spin_factor < 1 ||
      (p->precision != SGW_FP64 && p->precision != SGW_MIXED_FP32))
    return SGW_ERR_ARG;
  if (p->nao > 640 || p->naux > 640) return SGW_ERR_ARG;
  sgw_ctx* c = new sgw_ctx();
  c->p = *p;
  c->mats_f.assign(p->mats_f, p->mats_f + p->nw_f);
  c->mats_b.assign(p->mats_b, p->mats_b + p->nw_b);
  {
    // with frequency sets closed under w -> -w, G(tau), P0(tau), P(tau) and Sigma~(tau) keep the
    // Hermiticity of their inputs exactly, and the Gram stages may use it
    auto closed = [](const std::vector<int>& v, int shift) {
      for (int n : v)
        if (std::find(v.begin(), v.end(), -n - shift) == v.end()) return false;
      return true;
    };
    c->herm = closed(c->mats_f, 1) && closed(c->mats_b, 0);
  }
  c->p.mats_f = c->mats_f.data();
  c->p.mats_b = c->mats_b.data();
  c->Nk = p->nk[0] * p->nk[1] * p->nk[2];
  c->nao = p->nao;
  c->naux = p->naux;
  c->nt = p->ntau;
  c->nwf = p->nw_f;
  c->nwb = p->nw_b;
  if (cudaGetDevice(&c->device) != cudaSuccess) c->device = -1;
  sgw_status s = build_grid(c);
  if (s != SGW_OK) { delete c; return s; }
  auto upc = [&](double2*& d, const std::vector<cplx>& h) {
    std::vector<double2> t(h.size());
    for (size_t i = 0; i < h.size(); ++i) t[i] = make_double2(h[i].real(), h[i].imag());
    return upload(c, d, t);
  };
  std::vector<cplx> brow(c->beta_row.begin(), c->beta_row.end()), gli(c->gl_interp.begin(), c->gl_interp.end());
  if ((s = upc(c->d_TF, c->TF)) != SGW_OK || (s = upc(c->d_TFbar, c->TFbar)) != SGW_OK ||
      (s = upc(c->d_TB, c->TB)) != SGW_OK || (s = upc(c->d_TBbar, c->TBbar)) != SGW_OK ||
      (s = upc(c->d_beta_row, brow)) != SGW_OK || (s = upc(c->d_gl_interp, gli)) != SGW_OK ||
      (s = upload(c, c->d_nu_f, c->nu_f)) != SGW_OK || (s = upload(c, c->d_tau, c->tau)) != SGW_OK) {
    sgw_destroy(c);
    return s;
  }
  if (cudaMalloc(&c->d_status, sizeof(int)) != cudaSuccess || cudaMalloc(&c->d_scalar, 64 * sizeof(double)) != cudaSuccess ||
      cudaMalloc(&c->d_maxbits, 2 * sizeof(unsigned long long)) != cudaSuccess) {
    sgw_destroy(c);
    return SGW_ERR_OOM;
  }
  cudaMemset(c->d_status, 0, sizeof(int));
  cudaMemset(c->d_scalar, 0, 64 * sizeof(double));
  *out = c;
  return SGW_OK;
}

extern "C" SGW_API sgw_status sgw_destroy(sgw_ctx* c) {
  if (!c) return SGW_ERR_ARG;
  cudaDeviceSynchronize();
  dfree(c->d_TF); dfree(c->d_TFbar); dfree(c->d_TB); dfree(c->d_TBbar);
  dfree(c->d_beta_row); dfree(c->d_gl_interp); dfree(c->d_nu_f); dfree(c->d_tau);
  dfree(c->d_Uao); dfree(c->d_Uaux); dfree(c->d_refl); dfree(c->d_reflM); dfree(c->d_refl_tiles);
  dfree(c->d_ao_start); dfree(c->d_ao_size); dfree(c->d_ao_doff);
  dfree(c->d_aux_start); dfree(c->d_aux_size); dfree(c->d_aux_doff);
  dfree(c->d_full_start); dfree(c->d_full_size); dfree(c->d_full_doff);
  for (int b = 0; b < 2; ++b) { dfree(c->d_nunits[b]); dfree(c->d_units[b]); dfree(c->d_udoff[b]); }
  tc_free(c);
  dfree(c->d_V[0]); dfree(c->d_V[1]); dfree(c->d_V32[0]); dfree(c->d_V32[1]); dfree(c->d_H0); dfree(c->d_S);
  dfree(c->d_el_boff); dfree(c->d_el_eoff); dfree(c->d_el_bn); dfree(c->d_el_i); dfree(c->d_el_j); dfree(c->d_el_w);
  dfree(c->d_C0); dfree(c->d_eps0); dfree(c->d_epsw);
  free_plan(c->plan_p0); free_plan(c->plan_sigma); free_plan(c->plan_k); free_plan(c->plan_rho);
  free_plan(c->plan_p0_part); free_plan(c->plan_sigma_part);
  dfree(c->d_ws); dfree(c->d_g32); dfree(c->d_status); dfree(c->d_scalar); dfree(c->d_maxbits);
  dfree(c->d_w_items); dfree(c->d_dy_items); dfree(c->d_hf_tab); dfree(c->d_wh_items); dfree(c->d_wh_adj);
  for (auto& h : c->d_herm_items) dfree(h);
  for (auto& a : c->inv_aux)
    if (a) cudaStreamDestroy(a);
  for (auto& e : c->inv_ev)
    if (e) cudaEventDestroy(e);
  dfree(c->d_it_P0); dfree(c->d_it_P); dfree(c->d_it_S); dfree(c->d_it_H);
  if (c->h_pinned) cudaFreeHost(c->h_pinned);
  if (c->it_exec) cudaGraphExecDestroy(c->it_exec);
  if (c->it_graph) cudaGraphDestroy(c->it_graph);
  delete c;
  return SGW_OK;
}

extern "C" SGW_API sgw_status sgw_sync(sgw_ctx* c, sgw_stream stream) {
  if (!c) return SGW_ERR_ARG;
  CK(cudaStreamSynchronize(S(stream)));
  int st = 0;
  CK(cudaMemcpy(&st, c->d_status, sizeof(int), cudaMemcpyDeviceToHost));
  if (st == DEV_SINGULAR) {
    cudaMemset(c->d_status, 0, sizeof(int));
    return c->fail(SGW_ERR_SINGULAR, "zero pivot in a block inversion");
  }
  if (st == DEV_BADJOB) {
    cudaMemset(c->d_status, 0, sizeof(int));
    return c->fail(SGW_ERR_STATE, "a tensor-core job table entry failed its launch checks; results are invalid");
  }
  if (st == DEV_TIMEOUT) {
    cudaMemset(c->d_status, 0, sizeof(int));
    return c->fail(SGW_ERR_TIMEOUT, "a tensor-core pipeline wait ran out of time; its results are invalid");
  }
  return SGW_OK;
}

// ---------------------------------------------------------------------------
// a1: irrep basis
// ---------------------------------------------------------------------------
// tau reflection of P0 (Algorithm 3 loops tau to n_tau/2; here without its time reversal).  From
// Eq. (P0) with G(tau - beta) = -G(tau) and V^{k2,k1}_Q = (V^{k1,k2}_Q)^dagger,
//     P0^q(tau) = P0^{-q}(beta - tau)^T   (auxiliary basis, every q, every tau).
// On the Chebyshev roots beta - tau_j = tau_{n-1-j}.  In block coordinates, with U^k the rotated
// auxiliary basis of point k (P0^k = U^k P0_blk^{rep(k)} U^k^dagger), the wedge point w of q and
// the wedge point w' of -q:
//     P0_blk^w(tau) = M P0_blk^{w'}(beta - tau)^T M^dagger,   M = U^q^dagger conj(U^{-q}).
// M maps the blocks of w' onto those of w (both are irrep bases of the same little group); when it
// does so block by block for every wedge point, only the first ceil(n_tau/2) tau values are
// contracted and the rest follow from this relation.  SGW_P0_REFLECT=0 turns it off.
static sgw_status setup_p0_reflection(sgw_ctx* c) {
  c->refl_ok = false;
  c->n_refl = 0;
  c->n_refl_tiles = 0;
  dfree(c->d_refl);
  dfree(c->d_reflM);
  dfree(c->d_refl_tiles);
  const char* e = std::getenv("SGW_P0_REFLECT");
  if ((e && e[0] == '0') || c->nt < 2) return SGW_OK;
  const int n = c->naux, n1 = c->p.nk[0], n2 = c->p.nk[1], n3 = c->p.nk[2];
  const auto& U = c->hostU[1];  // [Nk][n][n], U[k][row][col]: column col is basis vector col
  auto kneg = [&](int k) {
    const int a = k / (n2 * n3), b = (k / n3) % n2, cc = k % n3;
    return (((n1 - a) % n1) * n2 + ((n2 - b) % n2)) * n3 + ((n3 - cc) % n3);
  };
  std::vector<ReflItem> items;
  std::vector<double2> Ms;
  std::vector<cplx> M((size_t)n * n);
  for (int w = 0; w < c->nwedge; ++w) {
    const int q = c->wedge_k[w], mq = kneg(q), w2 = c->rep[mq];
    const cplx* Uq = U.data() + (size_t)q * n * n;
    const cplx* Um = U.data() + (size_t)mq * n * n;
    // M[i][j] = sum_r conj(Uq[r][i]) conj(Um[r][j])
    std::fill(M.begin(), M.end(), cplx(0, 0));
    for (int r = 0; r < n; ++r)
      for (int i = 0; i < n; ++i) {
        const cplx a = std::conj(Uq[(size_t)r * n + i]);
        if (a == cplx(0, 0)) continue;
        const cplx* ur = Um + (size_t)r * n;
        cplx* mr = M.data() + (size_t)i * n;
        for (int j = 0; j < n; ++j) mr[j] += a * std::conj(ur[j]);
      }
    const Partition& Pt = c->part_aux[w];
    const Partition& Ps = c->part_aux[w2];
    std::vector<int> ss(Ps.sizes.size());
    for (size_t b = 0, s0 = 0; b < Ps.sizes.size(); s0 += Ps.sizes[b], ++b) ss[b] = (int)s0;
    int st = 0;
    long long doff = 0;
    for (int nb : Pt.sizes) {
      // the source block holding this row block's weight; everything else must vanish
      double best = -1.0, total = 0.0;
      int bb = -1;
      for (size_t b2 = 0; b2 < Ps.sizes.size(); ++b2) {
        double f = 0.0;
        for (int i = st; i < st + nb; ++i)
          for (int j = ss[b2]; j < ss[b2] + Ps.sizes[b2]; ++j) f += std::norm(M[(size_t)i * n + j]);
        total += f;
        if (f > best) { best = f; bb = (int)b2; }
      }
      // off-block elements of M at most about 1e-10 (they are rounding of the bases): else no reflection
      if (bb < 0 || Ps.sizes[bb] != nb || total - best > 1e-20 * (double)nb * n) return SGW_OK;
      long long soff = 0;
      for (int b2 = 0; b2 < bb; ++b2) soff += (long long)Ps.sizes[b2] * Ps.sizes[b2];
      items.push_back({c->p_off[w] + doff, c->p_off[w2] + soff, (long long)Ms.size(), nb, 0});
      for (int i = st; i < st + nb; ++i)
        for (int j = ss[bb]; j < ss[bb] + nb; ++j) {
          const cplx m = M[(size_t)i * n + j];
          Ms.push_back(make_double2(m.real(), m.imag()));
        }
      st += nb;
      doff += (long long)nb * nb;
    }
  }
  std::vector<ReflTile> tiles;
  for (size_t i = 0; i < items.size(); ++i) {
    const int nt32 = (items[i].n + 31) / 32;
    for (int ti = 0; ti < nt32; ++ti)
      for (int tj = 0; tj < nt32; ++tj) tiles.push_back({(int)i, ti, tj, 0});
  }
  CKS(upload(c, c->d_refl, items));
  CKS(upload(c, c->d_reflM, Ms));
  CKS(upload(c, c->d_refl_tiles, tiles));
  c->n_refl = (int)items.size();
  c->n_refl_tiles = (int)tiles.size();
  c->refl_ok = true;
  return SGW_OK;
}

int sgw::p0_tau_count(const sgw_ctx* c, long long pb, long long pe) {
  const bool whole = pb == 0 && pe == (long long)c->nwedge * c->Nk;
  return whole && c->refl_ok ? (c->nt + 1) / 2 : c->nt;
}

sgw_status sgw::p0_complete(sgw_ctx* c, double2* P0, int nt_eff, cudaStream_t st) {
  CKS(lower_from_upper(c, 1, P0, st));
  if (nt_eff >= c->nt) return SGW_OK;
  const size_t need = (size_t)(c->nt - nt_eff) * c->p_elems;
  CKS(ensure_workspace(c, need * sizeof(double2)));
  run(c, "p0_reflect", 0.0, 2, st, [&] {
    p0_reflect(c->d_refl, c->d_refl_tiles, c->n_refl_tiles, P0, c->p_elems, c->nt, nt_eff, c->d_reflM, c->d_ws, st);
  });
  return lower_from_upper(c, 1, P0, st);  // exactly Hermitian blocks (the products are, up to rounding)
}

extern "C" SGW_API sgw_status sgw_build_irrep_basis(sgw_ctx* c, const sgw_structure* st, sgw_layout* out) {
  if (!c || !st || !out) return SGW_ERR_ARG;
  if (st->natom < 1 || st->nops < 1 || !st->positions || !st->rotations || !st->translations || !st->ao_shells ||
      !st->aux_shells)
    return c->fail(SGW_ERR_ARG, "incomplete structure");
  CKS(build_symmetry(c, st));
  const int Nk = c->Nk, nao = c->nao, naux = c->naux, nw = c->nwedge;
  CKS(setup_p0_reflection(c));
  for (int b = 0; b < 2; ++b) {
    std::vector<double2> t(c->hostU[b].size());
    for (size_t i = 0; i < t.size(); ++i) t[i] = make_double2(c->hostU[b][i].real(), c->hostU[b][i].imag());
    CKS(upload(c, b == 0 ? c->d_Uao : c->d_Uaux, t));
    std::vector<sgw::cplx>().swap(c->hostU[b]);
  }
  // partition tables
  std::vector<int> s0, z0, s1, z1;
  std::vector<long long> d0, d1;
  for (int w = 0; w < nw; ++w) {
    s0.insert(s0.end(), c->part_ao[w].starts.begin(), c->part_ao[w].starts.end());
    z0.insert(z0.end(), c->part_ao[w].isize.begin(), c->part_ao[w].isize.end());
    d0.insert(d0.end(), c->part_ao[w].doff.begin(), c->part_ao[w].doff.end());
    s1.insert(s1.end(), c->part_aux[w].starts.begin(), c->part_aux[w].starts.end());
    z1.insert(z1.end(), c->part_aux[w].isize.begin(), c->part_aux[w].isize.end());
    d1.insert(d1.end(), c->part_aux[w].doff.begin(), c->part_aux[w].doff.end());
  }
  CKS(upload(c, c->d_ao_start, s0)); CKS(upload(c, c->d_ao_size, z0)); CKS(upload(c, c->d_ao_doff, d0));
  CKS(upload(c, c->d_aux_start, s1)); CKS(upload(c, c->d_aux_size, z1)); CKS(upload(c, c->d_aux_doff, d1));
  // chunked unit tables: every block split into runs of at most 8 outputs
  for (int b = 0; b < 2; ++b) {
    const auto& parts = b == 0 ? c->part_ao : c->part_aux;
    std::vector<std::vector<int4>> lists(nw);
    std::vector<std::vector<long long>> doffs(nw);
    int stride = 1;
    for (int w = 0; w < nw; ++w) {
      int st0 = 0;
      long long d0 = 0;
      for (int sz : parts[w].sizes) {
        for (int f = 0; f < sz; f += 8) {
          lists[w].push_back(make_int4(st0 + f, std::min(8, sz - f), st0, sz));
          doffs[w].push_back(d0);
        }
        st0 += sz;
        d0 += (long long)sz * sz;
      }
      stride = std::max(stride, (int)lists[w].size());
    }
    std::vector<int> nu(nw);
    std::vector<int4> un((size_t)nw * stride, make_int4(0, 0, 0, 1));
    std::vector<long long> ud((size_t)nw * stride, 0);
    for (int w = 0; w < nw; ++w) {
      nu[w] = (int)lists[w].size();
      std::copy(lists[w].begin(), lists[w].end(), un.begin() + (size_t)w * stride);
      std::copy(doffs[w].begin(), doffs[w].end(), ud.begin() + (size_t)w * stride);
    }
    CKS(upload(c, c->d_nunits[b], nu));
    CKS(upload(c, c->d_units[b], un));
    CKS(upload(c, c->d_udoff[b], ud));
    c->ustride[b] = stride;
  }
  const int W = std::max(nao, naux);
  std::vector<int> fs(2 * W, 0), fz(2 * W, 0);
  std::vector<long long> fd(2 * W, 0);
  for (int i = 0; i < W; ++i) { fz[i] = nao; fz[W + i] = naux; }
  CKS(upload(c, c->d_full_start, fs)); CKS(upload(c, c->d_full_size, fz)); CKS(upload(c, c->d_full_doff, fd));
  // block lists and per-element tables
  c->aob_off.clear(); c->aob_n.clear(); c->aob_w.clear(); c->aob_start.clear();
  c->auxb_off.clear(); c->auxb_n.clear(); c->auxb_w.clear(); c->auxb_start.clear();
  std::vector<long long> el_boff(c->g_elems), el_eoff(c->g_elems);
  std::vector<int> el_bn(c->g_elems), el_i(c->g_elems), el_j(c->g_elems), el_w(c->g_elems);
  for (int w = 0; w < nw; ++w) {
    long long off = c->g_off[w];
    int start = 0;
    for (int n : c->part_ao[w].sizes) {
      c->aob_off.push_back(off); c->aob_n.push_back(n); c->aob_w.push_back(w); c->aob_start.push_back(start);
      for (int a = 0; a < n; ++a)
        for (int b = 0; b < n; ++b) {
          const long long e = off + (long long)a * n + b;
          el_boff[e] = off; el_bn[e] = n; el_eoff[e] = (long long)w * nao + start;
          el_i[e] = start + a; el_j[e] = start + b; el_w[e] = w;
        }
      off += (long long)n * n;
      start += n;
    }
    off = c->p_off[w];
    start = 0;
    for (int n : c->part_aux[w].sizes) {
      c->auxb_off.push_back(off); c->auxb_n.push_back(n); c->auxb_w.push_back(w); c->auxb_start.push_back(start);
      off += (long long)n * n;
      start += n;
    }
  }
  CKS(upload(c, c->d_el_boff, el_boff)); CKS(upload(c, c->d_el_eoff, el_eoff)); CKS(upload(c, c->d_el_bn, el_bn));
  CKS(upload(c, c->d_el_i, el_i)); CKS(upload(c, c->d_el_j, el_j)); CKS(upload(c, c->d_el_w, el_w));
  // input storage
  const long long np = (long long)nw * Nk;
  for (int o = 0; o < 2; ++o) {
    dfree(c->d_V[o]);
    dfree(c->d_V32[o]);
    if (cudaMalloc(&c->d_V[o], (size_t)np * vsize(c) * sizeof(double2)) != cudaSuccess)
      return c->fail(SGW_ERR_OOM, "allocating the interaction tensor");
    if (c->p.precision == SGW_MIXED_FP32 &&
        cudaMalloc(&c->d_V32[o], (size_t)np * vsize(c) * sizeof(float2)) != cudaSuccess)
      return c->fail(SGW_ERR_OOM, "allocating the single-precision interaction tensor");
    c->have_v[o] = false;
    c->v_loaded[o].assign(np, 0);
  }
  dfree(c->d_H0); dfree(c->d_S);
  if (cudaMalloc(&c->d_H0, c->g_elems * sizeof(double2)) != cudaSuccess ||
      cudaMalloc(&c->d_S, c->g_elems * sizeof(double2)) != cudaSuccess)
    return c->fail(SGW_ERR_OOM, "allocating one-body blocks");
  free_plan(c->plan_p0); free_plan(c->plan_sigma); free_plan(c->plan_k); free_plan(c->plan_rho);
  free_plan(c->plan_p0_part); free_plan(c->plan_sigma_part);
  tc_free(c);
  c->use_tc = tc_supported(c);
  c->built = true;
  out->nkpts = Nk;
  out->nwedge = nw;
  out->g_elems = c->g_elems;
  out->p_elems = c->p_elems;
  out->npairs = np;
  out->max_ao_block = c->max_ao_block;
  out->max_aux_block = c->max_aux_block;
  return SGW_OK;
}

extern "C" SGW_API sgw_status sgw_get_wedge(const sgw_ctx* c, int* wedge_k, int* rep, int* op) {
  if (!c || !c->built) return SGW_ERR_STATE;
  if (wedge_k) std::copy(c->wedge_k.begin(), c->wedge_k.end(), wedge_k);
  if (rep) std::copy(c->rep.begin(), c->rep.end(), rep);
  if (op) std::copy(c->op.begin(), c->op.end(), op);
  return SGW_OK;
}

extern "C" SGW_API sgw_status sgw_get_blocks(const sgw_ctx* c, int which, int w, int* nblocks, int* sizes) {
  if (!c || !c->built) return SGW_ERR_STATE;
  if (w < 0 || w >= c->nwedge || (which != 0 && which != 1) || !nblocks) return SGW_ERR_ARG;
  const auto& P = which == 0 ? c->part_ao[w] : c->part_aux[w];
  *nblocks = (int)P.sizes.size();
  if (sizes) std::copy(P.sizes.begin(), P.sizes.end(), sizes);
  return SGW_OK;
}

extern "C" SGW_API sgw_status sgw_get_pairs(const sgw_ctx* c, int which, int* k1, int* k2) {
  if (!c || !c->built) return SGW_ERR_STATE;
  if (which != 0 && which != 1) return SGW_ERR_ARG;
  if (k1) std::copy(c->pair_k1[which].begin(), c->pair_k1[which].end(), k1);
  if (k2) std::copy(c->pair_k2[which].begin(), c->pair_k2[which].end(), k2);
  return SGW_OK;
}

extern "C" SGW_API sgw_status sgw_get_basis(const sgw_ctx* c0, int which, void* U, sgw_stream stream) {
  sgw_ctx* c = const_cast<sgw_ctx*>(c0);
  CKS(need_built(c));
  if (!U || (which != 0 && which != 1)) return SGW_ERR_ARG;
  const int n = which == 0 ? c->nao : c->naux;
  CK(cudaMemcpyAsync(U, which == 0 ? c->d_Uao : c->d_Uaux, (size_t)c->Nk * n * n * sizeof(double2),
                     cudaMemcpyDeviceToDevice, S(stream)));
  return SGW_OK;
}

// ---------------------------------------------------------------------------
// inputs
// ---------------------------------------------------------------------------
// dense per-wedge matrices [nw][n][n] -> U^dagger X U (left U^dagger, right U) -> packed diagonal blocks
static sgw_status block_one_body(sgw_ctx* c, const double2* src_bz, double2* dst_packed, cudaStream_t st) {
  const int nao = c->nao, nw = c->nwedge;
  const long long mat = (long long)nao * nao;
  CKS(ensure_workspace(c, (size_t)3 * nw * mat * sizeof(double2) + 4096));
  double2* A = c->d_ws;
  double2* B = A + nw * mat;
  for (int w = 0; w < nw; ++w)
    CK(cudaMemcpyAsync(A + w * mat, src_bz + (long long)c->wedge_k[w] * mat, mat * sizeof(double2),
                       cudaMemcpyDeviceToDevice, st));
  std::vector<BdItem> it(nw);
  for (int w = 0; w < nw; ++w) {
    it[w].x_off = w * mat;
    it[w].y_off = w * mat;
    it[w].m_off = (long long)c->wedge_k[w] * mat;
    it[w].part = 0;
    it[w].scale = z(1.0);
  }
  BdItem* d_it = reinterpret_cast<BdItem*>(B + nw * mat);
  CK(cudaMemcpyAsync(d_it, it.data(), nw * sizeof(BdItem), cudaMemcpyHostToDevice, st));
  const int W = std::max(c->nao, c->naux);
  const double fl1 = 8.0 * nw * (double)nao * nao * nao;
  run(c, "setup_rotate", fl1, 1, st, [&] {
    bd_mult(geom(1, nao, nao, 1, 1, 1, 0, W), A, B, c->d_Uao, d_it, nw, c->d_full_start, c->d_full_size,
            c->d_full_doff, st);
  });
  run(c, "setup_rotate", fl1, 1, st, [&] {
    bd_mult(geom(1, nao, nao, 0, 0, 0, 0, W), B, A, c->d_Uao, d_it, nw, c->d_full_start, c->d_full_size,
            c->d_full_doff, st);
  });
  std::vector<long long> bdo, bpo;
  std::vector<int> bn;
  for (size_t b = 0; b < c->aob_off.size(); ++b) {
    bdo.push_back(c->aob_w[b] * mat + (long long)c->aob_start[b] * nao + c->aob_start[b]);
    bpo.push_back(c->aob_off[b]);
    bn.push_back(c->aob_n[b]);
  }
  long long* d_bdo = reinterpret_cast<long long*>(d_it + nw);
  long long* d_bpo = d_bdo + bdo.size();
  int* d_bn = reinterpret_cast<int*>(d_bpo + bpo.size());
  CK(cudaMemcpyAsync(d_bdo, bdo.data(), bdo.size() * 8, cudaMemcpyHostToDevice, st));
  CK(cudaMemcpyAsync(d_bpo, bpo.data(), bpo.size() * 8, cudaMemcpyHostToDevice, st));
  CK(cudaMemcpyAsync(d_bn, bn.data(), bn.size() * 4, cudaMemcpyHostToDevice, st));
  run(c, "pack", 0.0, 1, st, [&] { pack_blocks(A, mat, nao, d_bdo, d_bn, d_bpo, (int)bn.size(), dst_packed, 1, st); });
  CK(cudaStreamSynchronize(st));
  return SGW_OK;
}

extern "C" SGW_API sgw_status sgw_load_one_body(sgw_ctx* c, const void* H0, const void* Sm, sgw_stream stream) {
  CKS(need_built(c));
  if (!H0 || !Sm) return c->fail(SGW_ERR_ARG, "null input");
  CKS(block_one_body(c, static_cast<const double2*>(H0), c->d_H0, S(stream)));
  CKS(block_one_body(c, static_cast<const double2*>(Sm), c->d_S, S(stream)));
  c->have_one_body = true;
  return SGW_OK;
}

extern "C" SGW_API sgw_status sgw_load_v(sgw_ctx* c, int which, long long first, long long count, const void* V,
                                         sgw_stream stream) {
  CKS(need_built(c));
  const long long np = (long long)c->nwedge * c->Nk;
  if ((which != 0 && which != 1) || !V || first < 0 || count < 1 || first + count > np)
    return c->fail(SGW_ERR_ARG, "sgw_load_v: bad pair range");
  cudaStream_t st = S(stream);
  const int nao = c->nao, naux = c->naux, Nk = c->Nk;
  const long long vs = vsize(c);
  const int W = std::max(nao, naux);
  // process in pieces that fit the workspace: two intermediates of the piece
  const size_t budget = workspace_budget();
  long long piece = std::max(1LL, (long long)(budget / (2 * vs * sizeof(double2) + 1)));
  piece = std::min(piece, count);
  CKS(ensure_workspace(c, (size_t)2 * piece * vs * sizeof(double2) + (size_t)3 * piece * sizeof(BdItem) + 4096));
  double2* Y = c->d_ws;
  double2* Z = Y + piece * vs;
  BdItem* d_items = reinterpret_cast<BdItem*>(Z + piece * vs);
  const double2* Vin = static_cast<const double2*>(V);
  for (long long p0 = 0; p0 < count; p0 += piece) {
    const long long np_ = std::min(piece, count - p0);
    std::vector<BdItem> ia(np_), ib(np_), ic(np_);
    for (long long i = 0; i < np_; ++i) {
      const long long p = first + p0 + i;
      const int k1 = c->pair_k1[which][p], k2 = c->pair_k2[which][p];
      // aux momentum q = k2 - k1 (orientation 0, basis U^q, rows conj(U)^T) or q = k1 - k2 (orientation 1, basis
      // conj(U^{k1-k2}): rows U^T)
      int qa;
      {
        const int n1 = c->p.nk[0], n2 = c->p.nk[1], n3 = c->p.nk[2];
        auto iv = [&](int k, int d) { return d == 0 ? k / (n2 * n3) : d == 1 ? (k / n3) % n2 : k % n3; };
        int a = iv(k2, 0) - iv(k1, 0), b = iv(k2, 1) - iv(k1, 1), cc = iv(k2, 2) - iv(k1, 2);
        if (which == 1) { a = -a; b = -b; cc = -cc; }
        a = ((a % n1) + n1) % n1; b = ((b % n2) + n2) % n2; cc = ((cc % n3) + n3) % n3;
        qa = (a * n2 + b) * n3 + cc;
      }
      ia[i] = {i * vs, i * vs, (long long)qa * naux * naux, 1, 0, z(1.0)};
      ib[i] = {i * vs, i * vs, (long long)k1 * nao * nao, 0, 0, z(1.0)};
      ic[i] = {i * vs, (p)*vs, (long long)k2 * nao * nao, 0, 0, z(1.0)};
    }
    CK(cudaMemcpyAsync(d_items, ia.data(), np_ * sizeof(BdItem), cudaMemcpyHostToDevice, st));
    CK(cudaMemcpyAsync(d_items + np_, ib.data(), np_ * sizeof(BdItem), cudaMemcpyHostToDevice, st));
    CK(cudaMemcpyAsync(d_items + 2 * np_, ic.data(), np_ * sizeof(BdItem), cudaMemcpyHostToDevice, st));
    // aux: Y[A][(c,d)] = sum_Q L[A][Q] V[Q][(c,d)], L = conj(U^q)^T (which 0) or (U^q)^T (which 1)
    const double fla = 8.0 * np_ * (double)naux * naux * nao * nao, flo = 8.0 * np_ * (double)naux * nao * nao * nao;
    run(c, "setup_rotate", fla, 1, st, [&] {
      bd_mult(geom(1, naux, nao * nao, 1, 1, which == 0 ? 1 : 0, 0, W), Vin + p0 * vs, Y, c->d_Uaux, d_items, np_,
              c->d_full_start, c->d_full_size, c->d_full_doff, st);
    });
    // left orbital: Z[A][i][d] = sum_c conj(U^{k1}[c][i]) Y[A][c][d]
    run(c, "setup_rotate", flo, 1, st, [&] {
      bd_mult(geom(naux, nao, nao, 1, 1, 1, 0, W), Y, Z, c->d_Uao, d_items + np_, np_, c->d_full_start,
              c->d_full_size, c->d_full_doff, st);
    });
    // right orbital: V_blk[A][i][j] = sum_d Z[A][i][d] U^{k2}[d][j]
    run(c, "setup_rotate", flo, 1, st, [&] {
      bd_mult(geom(naux, nao, nao, 0, 0, 0, 0, W), Z, c->d_V[which], c->d_Uao, d_items + 2 * np_, np_,
              c->d_full_start, c->d_full_size, c->d_full_doff, st);
    });
    if (c->p.precision == SGW_MIXED_FP32) {
      const long long pbeg = first + p0;
      run(c, "convert", 0.0, 1, st, [&] {
        if (c->use_tc)
          tc_store_v(c, which, c->d_V[which] + pbeg * vs, c->d_V32[which] + pbeg * vs, np_, st);
        else
          to_c64(c->d_V[which] + pbeg * vs, c->d_V32[which] + pbeg * vs, np_ * vs, st);
      });
    }
    CK(cudaStreamSynchronize(st));
    for (long long i = 0; i < np_; ++i) c->v_loaded[which][first + p0 + i] = 1;
  }
  (void)Nk;
  c->have_v[which] = std::all_of(c->v_loaded[which].begin(), c->v_loaded[which].end(), [](long long x) { return x; });
  return SGW_OK;
}

// ---------------------------------------------------------------------------
// G0 and mu0
// ---------------------------------------------------------------------------
extern "C" SGW_API sgw_status sgw_g0(sgw_ctx* c, double* mu_out, void* G_tau, sgw_stream stream) {
  CKS(need_built(c));
  if (!c->have_one_body) return c->fail(SGW_ERR_STATE, "one-body inputs not loaded");
  if (!mu_out || !G_tau) return SGW_ERR_ARG;
  cudaStream_t st = S(stream);
  const int nao = c->nao, nw = c->nwedge;
  if (!c->d_C0) {
    if (cudaMalloc(&c->d_C0, c->g_elems * sizeof(double2)) != cudaSuccess ||
        cudaMalloc(&c->d_eps0, (size_t)nw * nao * sizeof(double)) != cudaSuccess ||
        cudaMalloc(&c->d_epsw, (size_t)nw * nao * sizeof(double)) != cudaSuccess)
      return c->fail(SGW_ERR_OOM, "allocating eigenpairs");
  }
  std::vector<EigItem> items;
  for (size_t b = 0; b < c->aob_off.size(); ++b)
    items.push_back({c->aob_off[b], c->aob_off[b], c->aob_off[b],
                     (long long)c->aob_w[b] * nao + c->aob_start[b], c->aob_n[b], 0});
  const int maxn = c->max_ao_block;
  const int grid = std::min<int>((int)items.size(), 304);
  CKS(ensure_workspace(c, (size_t)grid * 4 * maxn * maxn * sizeof(double2) + items.size() * sizeof(EigItem) + 4096));
  EigItem* d_items = reinterpret_cast<EigItem*>(c->d_ws + (size_t)grid * 4 * maxn * maxn);
  CK(cudaMemcpyAsync(d_items, items.data(), items.size() * sizeof(EigItem), cudaMemcpyHostToDevice, st));
  double fle = 0;
  for (auto& it : items) fle += 3 * 8.0 * it.n * it.n * it.n;
  run(c, "eigh", fle, 1, st, [&] { geneig(d_items, (int)items.size(), maxn, c->d_H0, c->d_S, c->d_C0, c->d_eps0, c->d_ws, st); });
  std::vector<double> wts((size_t)nw * nao);
  for (int w = 0; w < nw; ++w)
    for (int i = 0; i < nao; ++i) wts[(size_t)w * nao + i] = (double)c->p.spin_factor / c->Nk * c->star[w];
  CK(cudaMemcpyAsync(c->d_epsw, wts.data(), wts.size() * sizeof(double), cudaMemcpyHostToDevice, st));
  double mu = 0.0;
  run(c, "mu_bisect", 0.0, 1, st, [&] {
    mu = mu_bisect_device(c->d_eps0, c->d_epsw, nw * nao, c->p.beta, c->p.n_elec, -60.0, 60.0, c->d_scalar, st);
  });
  run(c, "g0", 0.0, 1, st, [&] {
    g0_closed_form(c->d_C0, c->d_eps0, c->d_el_boff, c->d_el_bn, c->d_el_eoff, c->g_elems, c->d_tau, c->nt,
                   c->p.beta, mu, static_cast<double2*>(G_tau), st);
  });
  CK(cudaGetLastError());
  *mu_out = mu;
  return SGW_OK;
}

// ---------------------------------------------------------------------------
// a3: polarization
// ---------------------------------------------------------------------------
// With Hermitian G^k(tau) and V^{k2,k1}_Q = (V^{k1,k2}_Q)^dagger, every block of P0^q(tau)
// (Eq. (P0)) is Hermitian, and with it P^q(tau) and Sigma~^k(tau) (Eqs. (P02P), (sigma)) when
// the frequency sets are closed under w -> -w (c->herm).  The Gram stages then contract only the
// tiles on and above the diagonal, and this fills the strict lower triangle of every block of the
// family (which = 0: Sigma~, orbital blocks at every tau; 1: P0, auxiliary blocks at every tau;
// 2: Sigma_HF, orbital blocks, one matrix per wedge point) by conjugate transposition.  Without
// c->herm the Gram stages contract every tile and nothing is filled.
double sgw::gram_elems(const sgw_ctx* c, int nb) { return c->herm ? 0.5 * nb * (nb + 1.0) : (double)nb * nb; }

// Block table of a family (which as in lower_from_upper), built on first use.
static sgw_status herm_items(sgw_ctx* c, int which) {
  HermItem*& d = c->d_herm_items[which];
  int& n = c->n_herm_items[which];
  if (d) return SGW_OK;
  const auto& off = which == 1 ? c->auxb_off : c->aob_off;
  const auto& sz = which == 1 ? c->auxb_n : c->aob_n;
  const long long elems = which == 1 ? c->p_elems : c->g_elems;
  const int nmat = which == 2 ? 1 : c->nt;  // Sigma_HF has no tau axis
  std::vector<HermItem> h;
  for (int t = 0; t < nmat; ++t)
    for (size_t b = 0; b < off.size(); ++b) h.push_back({(long long)t * elems + off[b], sz[b], 0});
  n = (int)h.size();
  if (h.empty()) return SGW_OK;
  return upload(c, d, h);
}

sgw_status sgw::lower_from_upper(sgw_ctx* c, int which, double2* X, cudaStream_t st) {
  if (!c->herm) return SGW_OK;
  CKS(herm_items(c, which));
  const HermItem* d = c->d_herm_items[which];
  const int n = c->n_herm_items[which];
  run(c, which == 0 ? "sigma_mirror" : which == 1 ? "p0_mirror" : "hf_mirror", 0.0, 1, st,
      [&] { hermitian_fill(d, n, X, st); });
  return SGW_OK;
}

// G(tau) of Eq. (dyson) is Hermitian at every tau when H0, S, Sigma_HF and Sigma~(tau) are and the
// fermionic set is closed under w -> -w: with c->herm the Dyson output is replaced
// by its Hermitian part, which changes it only at the rounding level and keeps the loop on the
// Hermitian subspace (an anti-Hermitian rounding component is otherwise free to grow from pass to
// pass in an undamped loop).
static sgw_status hermitian_g(sgw_ctx* c, double2* G, cudaStream_t st) {
  if (!c->herm) return SGW_OK;
  CKS(herm_items(c, 0));
  const HermItem* d = c->d_herm_items[0];
  const int n = c->n_herm_items[0];
  run(c, "g_hermitian", 0.0, 1, st, [&] { hermitian_part(d, n, G, st); });
  return SGW_OK;
}

// Plans of the block-multiply / Gram chains cover the pairs [pb, pe) of their orientation's pair
// list (ordered [wedge point][k]); the intermediates are indexed by the local pair p - pb.
static sgw_status build_p0_plan(sgw_ctx* c, ContractionPlan& P, long long pb, long long pe) {
  if (P.built && P.pb == pb && P.pe == pe) return SGW_OK;
  free_plan(P);
  P.pb = pb;
  P.pe = pe;
  const int Nk = c->Nk, nt = c->nt, nao = c->nao;
  const int nte = p0_tau_count(c, pb, pe);  // tau values contracted; the rest by the reflection
  P.nt_eff = nte;
  const long long vs = vsize(c), np = pe - pb;
  const size_t budget = workspace_budget();
  int nc = (int)std::max<long long>(1, (long long)(budget * 0.8 / (2.0 * np * vs * sizeof(double2))));
  nc = std::min(nc, nte);
  P.nc = nc;
  P.items_per_t = np;
  std::vector<BdItem> A((size_t)nte * np), B((size_t)nte * np);
  for (int t = 0; t < nte; ++t) {
    const int tl = t % nc;
    for (long long lp = 0; lp < np; ++lp) {
      const long long p = pb + lp;
      const int k1 = c->pair_k1[0][p], k2 = c->pair_k2[0][p];
      const long long pos = (lp * nc + tl) * vs;
      BdItem a;
      a.x_off = p * vs;
      a.y_off = pos;
      a.m_off = (long long)t * c->g_elems + c->g_off[c->rep[k2]];
      a.part = c->rep[k2];
      a.pad = 0;
      a.scale = z(1.0);
      A[(size_t)t * np + lp] = a;
      BdItem b;
      b.x_off = pos;
      b.y_off = pos;
      b.m_off = (long long)(nt - 1 - t) * c->g_elems + c->g_off[c->rep[k1]];
      b.part = c->rep[k1];
      b.pad = 0;
      b.scale = z(-1.0);  // G(-tau_j) = -G(tau_{n-1-j})
      B[(size_t)t * np + lp] = b;
    }
  }
  std::vector<GramUnit> units;
  std::vector<GramTile> tiles;
  P.unit_start.assign(nt + 1, 0);
  P.tile_start.assign(nt + 1, 0);
  long long base = 0;
  double work_t = 0;
  for (size_t b = 0; b < c->auxb_off.size(); ++b) work_t += (double)c->auxb_n[b] * c->auxb_n[b] * nao * nao * Nk;
  const long long target = unit_target(work_t * nc);
  for (int t = 0; t < nte; ++t) {
    if (t % nc == 0) {
      if (t > 0) schedule_units(units, (size_t)base, 0);
      base = (long long)units.size();
    }
    P.unit_start[t] = units.size();
    P.tile_start[t] = tiles.size();
    const int tl = t % nc;
    for (size_t b = 0; b < c->auxb_off.size(); ++b) {
      const int w = c->auxb_w[b], nb = c->auxb_n[b], st = c->auxb_start[b];
      // the pairs of wedge point w inside the range (none: the block stays zero)
      const long long p0 = std::max(pb, (long long)w * Nk), p1 = std::min(pe, (long long)(w + 1) * Nk);
      if (p1 <= p0) continue;
      const size_t from = units.size();
      add_gram_block(units, tiles, base, nb, (long long)t * c->p_elems + c->auxb_off[b],
                     ((p0 - pb) * nc + tl) * vs + (long long)st * nao * nao, p0 * vs + (long long)st * nao * nao,
                     (long long)nao * nao, (long long)nao * nao, (int)(p1 - p0), (long long)nao * nao, target,
                     c->herm);
      finalize_units(units, from, (long long)nc * vs, vs);
    }
  }
  schedule_units(units, (size_t)base, 0);
  for (int t = nte; t <= nt; ++t) {
    P.unit_start[t] = units.size();
    P.tile_start[t] = tiles.size();
  }
  P.max_units_chunk = 0;
  for (int t0 = 0; t0 < nte; t0 += nc) {
    const int t1 = std::min(nte, t0 + nc);
    P.max_units_chunk = std::max(P.max_units_chunk, P.unit_start[t1] - P.unit_start[t0]);
  }
  P.fl_A_t = P.fl_B_t = P.fl_G_t = 0;
  for (long long p = pb; p < pe; ++p) {
    P.fl_A_t += 8.0 * c->naux * nao * (double)c->part_ao[c->rep[c->pair_k2[0][p]]].elems;
    P.fl_B_t += 8.0 * c->naux * nao * (double)c->part_ao[c->rep[c->pair_k1[0][p]]].elems;
  }
  // with Hermitian blocks the Gram stage needs their upper triangles only
  for (size_t b = 0; b < c->auxb_n.size(); ++b) {
    const int w = c->auxb_w[b];
    const long long npw = std::max(0LL, std::min(pe, (long long)(w + 1) * Nk) - std::max(pb, (long long)w * Nk));
    P.fl_G_t += 8.0 * npw * (double)nao * nao * gram_elems(c, c->auxb_n[b]);
  }
  CKS(upload(c, P.d_A, A));
  CKS(upload(c, P.d_B, B));
  CKS(upload(c, P.d_units, units));
  CKS(upload(c, P.d_tiles, tiles));
  P.built = true;
  return SGW_OK;
}

template <typename Z>
static sgw_status polarization_impl(sgw_ctx* c, const ContractionPlan& P, const Z* G, const Z* V, double2* out,
                                    cudaStream_t st, const char* tag) {
  const int nt = c->nt, nao = c->nao, naux = c->naux, nc = P.nc;
  const long long vs = vsize(c), np = P.items_per_t;
  const size_t inter = (size_t)np * nc * vs;
  const size_t gsz = std::is_same<Z, float2>::value ? (size_t)nt * c->g_elems : 0;
  CKS(ensure_workspace(c, (2 * inter + (size_t)P.max_units_chunk * 1024 + gsz) * sizeof(Z)));
  Z* Zw = reinterpret_cast<Z*>(c->d_ws);
  Z* X = Zw + inter;
  Z* part = X + inter;
  GramGeom gg;
  gg.a_pair = (long long)nc * vs;
  gg.b_pair = vs;
  gg.a_row = (long long)nao * nao;
  gg.b_row = (long long)nao * nao;
  gg.k_outer_a = 0;
  gg.k_outer_b = 0;
  gg.k_inner = nao * nao;
  gg.k_outer = 1;
  const double alpha = c->p.loop_sign * (double)c->p.spin_factor / c->Nk;
  const std::string t_vg = std::string("p0_vg") + tag, t_gvg = std::string("p0_gvg") + tag,
                    t_gram = std::string("p0_gram") + tag;
  for (int t0 = 0; t0 < P.nt_eff; t0 += nc) {
    const int t1 = std::min(P.nt_eff, t0 + nc);
    const long long ni = (long long)(t1 - t0) * np;
    const int ntc = t1 - t0;
    // Z[A][c][j] = sum_d V[A][c][d] G^{k+q}(tau)[d][j]
    run(c, t_vg.c_str(), P.fl_A_t * ntc, 1, st, [&] {
      bdm(c, 0, geom(1, naux * nao, nao, 0, 0, 0, 0, nao), V, Zw, G, P.d_A + (size_t)t0 * np, ni, st);
    });
    // X[A][i][j] = sum_c G^k(-tau)[i][c] Z[A][c][j]
    run(c, t_gvg.c_str(), P.fl_B_t * ntc, 1, st, [&] {
      bdm(c, 0, geom(naux, nao, nao, 1, 0, 0, 0, nao), Zw, X, G, P.d_B + (size_t)t0 * np, ni, st);
    });
    const long long u0 = P.unit_start[t0], u1 = P.unit_start[t1];
    const long long ti0 = P.tile_start[t0], ti1 = P.tile_start[t1];
    run(c, t_gram.c_str(), P.fl_G_t * ntc, 1, st, [&] { gram_partials(gg, X, V, P.d_units + u0, (int)(u1 - u0), part, st); });
    run(c, "gram_reduce", 0.0, 1, st, [&] { gram_reduce(P.d_tiles + ti0, (int)(ti1 - ti0), part, out, z(alpha), 0, st); });
  }
  return p0_complete(c, out, P.nt_eff, st);
}

static sgw_status polarization_range(sgw_ctx* c, const void* G_tau, void* P0_tau, long long pb, long long pe,
                                     sgw_stream stream) {
  CKS(need_built(c));
  if (!c->have_v[0]) return c->fail(SGW_ERR_STATE, "polarization pairs of V not loaded");
  const long long np = (long long)c->nwedge * c->Nk;
  if (!G_tau || !P0_tau || pb < 0 || pe > np || pb > pe) return SGW_ERR_ARG;
  const bool whole = pb == 0 && pe == np;
  cudaStream_t st = S(stream);
  double2* out = static_cast<double2*>(P0_tau);
  // blocks of wedge points without pairs in a partial range are not written by the chains
  if (!whole) CK(cudaMemsetAsync(out, 0, (size_t)c->nt * c->p_elems * sizeof(double2), st));
  if (pb == pe) return SGW_OK;  // an empty range: the partial sum is zero
  ContractionPlan& P = whole ? c->plan_p0 : c->plan_p0_part;
  if (!c->use_tc) CKS(build_p0_plan(c, P, pb, pe));
  if (c->use_tc) {
    // tensor-core chains: TF32 head/tail products, FP32 accumulation, FP64 sums of the partial tiles
    CKS(tc_polarization(c, static_cast<const double2*>(G_tau), out, pb, pe, st));
  } else if (c->p.precision == SGW_MIXED_FP32) {
    // G(tau) rounded to complex64 once; the chains accumulate in FP32, P0 is returned in FP64
    CKS(ensure_g32(c, (size_t)c->nt * c->g_elems));
    run(c, "convert", 0.0, 1, st, [&] { to_c64(static_cast<const double2*>(G_tau), c->d_g32, (long long)c->nt * c->g_elems, st); });
    CKS(polarization_impl<float2>(c, P, c->d_g32, c->d_V32[0], out, st, "_f32"));
  } else {
    CKS(polarization_impl<double2>(c, P, static_cast<const double2*>(G_tau), c->d_V[0], out, st, ""));
  }
  CK(cudaGetLastError());
  return SGW_OK;
}

extern "C" SGW_API sgw_status sgw_polarization(sgw_ctx* c, const void* G_tau, void* P0_tau, sgw_stream stream) {
  if (!c) return SGW_ERR_ARG;
  return polarization_range(c, G_tau, P0_tau, 0, (long long)c->nwedge * c->Nk, stream);
}

extern "C" SGW_API sgw_status sgw_polarization_pairs(sgw_ctx* c, const void* G_tau, void* P0_tau, long long pair_begin,
                                                     long long pair_end, sgw_stream stream) {
  if (!c) return SGW_ERR_ARG;
  return polarization_range(c, G_tau, P0_tau, pair_begin, pair_end, stream);
}

// ---------------------------------------------------------------------------
// static launch tables of the hot path
// ---------------------------------------------------------------------------
static sgw_status ensure_tables(sgw_ctx* c) {
  if (c->tables) return SGW_OK;
  std::vector<InvItem> w;
  for (int m = 0; m < c->nwb; ++m)
    for (size_t b = 0; b < c->auxb_off.size(); ++b) {
      InvItem it;
      it.a_off = (long long)m * c->p_elems + c->auxb_off[b];
      it.s_off = it.f_off = 0;
      it.out_off = it.a_off;
      it.n = c->auxb_n[b];
      it.m = m;
      it.weight = z(0.0);
      w.push_back(it);
    }
  // With a bosonic set closed under n -> -n and sorted, the W blocks at -Omega_n are the adjoints of
  // those at Omega_n (P0(tau) blocks are Hermitian, so P0(-i Omega) = P0(i Omega)^dagger, and W
  // inherits it): only rows [wh_m0, nw_b) are solved, each row m < wh_m0 is the adjoint of row
  // nw_b - 1 - m.
  std::vector<InvItem> wh;
  std::vector<AdjItem> adj;
  c->wh_m0 = -1;
  {
    bool sym = c->herm;
    for (int m = 0; m < c->nwb && sym; ++m)
      sym = c->mats_b[c->nwb - 1 - m] == -c->mats_b[m] && (m == 0 || c->mats_b[m] > c->mats_b[m - 1]);
    if (sym) {
      int m0 = 0;
      while (m0 < c->nwb && c->mats_b[m0] < 0) ++m0;
      c->wh_m0 = m0;
      for (const InvItem& it : w)
        if (it.m >= m0) wh.push_back(it);
      for (int m = 0; m < m0; ++m)
        for (size_t b = 0; b < c->auxb_off.size(); ++b) {
          AdjItem a;
          a.src_off = (long long)(c->nwb - 1 - m) * c->p_elems + c->auxb_off[b];
          a.dst_off = (long long)m * c->p_elems + c->auxb_off[b];
          a.n = c->auxb_n[b];
          a.pad = 0;
          adj.push_back(a);
        }
    }
  }
  std::vector<InvItem> d;
  for (int m = 0; m < c->nwf; ++m)
    for (size_t b = 0; b < c->aob_off.size(); ++b) {
      InvItem it;
      it.a_off = (long long)m * c->g_elems + c->aob_off[b];
      it.s_off = c->aob_off[b];
      it.f_off = c->aob_off[b];
      it.out_off = it.a_off;
      it.n = c->aob_n[b];
      it.m = m;
      const double wk = (double)c->p.spin_factor / c->Nk * c->star[c->aob_w[b]];
      it.weight = z(wk * c->gamma_w[m].real(), wk * c->gamma_w[m].imag());
      d.push_back(it);
    }
  const size_t nb = c->aob_off.size();
  const long long mat = (long long)c->nao * c->nao, vs = vsize(c);
  std::vector<long long> tab(3 * nb + c->nwedge);
  for (size_t b = 0; b < nb; ++b) {
    tab[b] = c->aob_w[b] * mat + (long long)c->aob_start[b] * c->nao + c->aob_start[b];
    tab[nb + b] = c->aob_off[b];
  }
  int* bn = reinterpret_cast<int*>(tab.data() + 2 * nb);
  for (size_t b = 0; b < nb; ++b) bn[b] = c->aob_n[b];
  const int wG = c->rep[0];
  for (int w = 0; w < c->nwedge; ++w) tab[3 * nb + w] = ((long long)wG * c->Nk + c->wedge_k[w]) * vs;
  // three groups (warp-sized blocks, blocks above 90 in global scratch, the rest in shared
  // memory); the two CTA groups ordered largest first so the longest eliminations start first,
  // the warp group left in frequency order (eight warps of a CTA share one SM's FP64 pipe, so
  // its CTAs are best mixed in size); slots keep the original order so the trace partials are
  // summed in a fixed order
  auto group = [](const InvItem& x) { return x.n <= 32 ? 0 : x.n > 90 ? 1 : 2; };
  auto split = [&](std::vector<InvItem>& v, InvPlan& pl) {
    for (size_t i = 0; i < v.size(); ++i) v[i].slot = (int)i;
    std::stable_sort(v.begin(), v.end(), [&](const InvItem& a, const InvItem& b) {
      const int ga = group(a), gb = group(b);
      return ga != gb ? ga < gb : (ga != 0 && a.n > b.n);
    });
    pl = InvPlan();
    pl.nitems = (int)v.size();
    for (auto& x : v) {
      const int g = group(x);
      if (g == 0) { ++pl.nsmall; pl.small_n = std::max(pl.small_n, x.n); }
      else if (g == 1) ++pl.nscr;
      else pl.mid_n = std::max(pl.mid_n, x.n);
      pl.max_n = std::max(pl.max_n, x.n);
    }
  };
  split(w, c->w_plan);
  split(d, c->dy_plan);
  if (c->wh_m0 >= 0) {
    split(wh, c->wh_plan);
    CKS(upload(c, c->d_wh_items, wh));
    CKS(upload(c, c->d_wh_adj, adj));
    c->n_wh_adj = (int)adj.size();
  }
  if (c->w_plan.max_n > 1024 || c->dy_plan.max_n > 1024)
    return c->fail(SGW_ERR_ARG, "irrep blocks above 1024 are not supported by the inversion kernels");
  CKS(upload(c, c->d_w_items, w));
  CKS(upload(c, c->d_dy_items, d));
  CKS(upload(c, c->d_hf_tab, tab));
  c->n_w_items = (int)w.size();
  c->n_dy_items = (int)d.size();
  if (!c->inv_aux[0]) {
    for (int i = 0; i < 2; ++i) CK(cudaStreamCreateWithFlags(&c->inv_aux[i], cudaStreamNonBlocking));
    for (int i = 0; i < 3; ++i) CK(cudaEventCreateWithFlags(&c->inv_ev[i], cudaEventDisableTiming));
  }
  for (InvPlan* pl : {&c->w_plan, &c->dy_plan, &c->wh_plan}) {
    pl->aux[0] = c->inv_aux[0];
    pl->aux[1] = c->inv_aux[1];
    pl->fork = c->inv_ev[0];
    pl->join[0] = c->inv_ev[1];
    pl->join[1] = c->inv_ev[2];
  }
  c->w_plan.items = c->d_w_items;
  c->dy_plan.items = c->d_dy_items;
  c->wh_plan.items = c->d_wh_items;
  c->tables = true;
  return SGW_OK;
}

// ---------------------------------------------------------------------------
// a4-a6: screened interaction
// ---------------------------------------------------------------------------
extern "C" SGW_API sgw_status sgw_screened_interaction(sgw_ctx* c, const void* P0_tau, void* P_tau, sgw_stream stream) {
  CKS(need_built(c));
  if (!P0_tau || !P_tau) return SGW_ERR_ARG;
  CKS(ensure_tables(c));
  cudaStream_t st = S(stream);
  const long long pe = c->p_elems;
  const int maxn = c->max_aux_block;
  const size_t wbytes = (size_t)2 * c->nwb * pe * sizeof(double2);
  const size_t scratch = maxn > 90 ? (size_t)304 * maxn * maxn * sizeof(double2) : 0;
  CKS(ensure_workspace(c, wbytes + scratch + 4096));
  double2* P0w = c->d_ws;
  double2* Pw = P0w + (size_t)c->nwb * pe;
  double2* scr = Pw + (size_t)c->nwb * pe;
  const double flt = 8.0 * c->nwb * (double)c->nt * pe;
  // rows [m0, nw_b) are transformed and solved; with the adjoint relation the rest are filled
  const int m0 = c->wh_m0 >= 0 ? c->wh_m0 : 0, nsolve = c->nwb - m0;
  const InvPlan& wp = c->wh_m0 >= 0 ? c->wh_plan : c->w_plan;
  double flw = 0;
  for (size_t b = 0; b < c->auxb_n.size(); ++b) flw += 8.0 * nsolve * std::pow((double)c->auxb_n[b], 3);
  run(c, "ft", 8.0 * nsolve * (double)c->nt * pe, 1, st, [&] {
    series_map(c->d_TB + (size_t)m0 * c->nt, nsolve, c->nt, static_cast<const double2*>(P0_tau), pe,
               P0w + (size_t)m0 * pe, pe, pe, z(1.0), 0, st);
  });
  run(c, "w_solve", flw, 1, st, [&] {
    invert_plan(INV_W, wp, P0w, nullptr, nullptr, nullptr, 0.0, nullptr, nullptr, Pw, nullptr, scr, c->d_status, st);
  });
  if (c->wh_m0 > 0)
    run(c, "w_mirror", 0.0, 1, st, [&] { block_adjoint(c->d_wh_adj, c->n_wh_adj, Pw, st); });
  run(c, "ft", flt, 1, st, [&] {
    series_map(c->d_TBbar, c->nt, c->nwb, Pw, pe, static_cast<double2*>(P_tau), pe, pe, z(1.0), 0, st);
  });
  CK(cudaGetLastError());
  return SGW_OK;
}

// ---------------------------------------------------------------------------
// a7: self-energy
// ---------------------------------------------------------------------------
static sgw_status build_sigma_plan(sgw_ctx* c, ContractionPlan& P, long long pb, long long pe) {
  if (P.built && P.pb == pb && P.pe == pe) return SGW_OK;
  free_plan(P);
  P.pb = pb;
  P.pe = pe;
  const int Nk = c->Nk, nt = c->nt, nao = c->nao;
  const long long vs = vsize(c), np = pe - pb;
  const size_t budget = workspace_budget();
  int nc = (int)std::max<long long>(1, (long long)(budget * 0.8 / (2.0 * np * vs * sizeof(double2))));
  nc = std::min(nc, nt);
  P.nc = nc;
  P.items_per_t = np;
  const int n1 = c->p.nk[0], n2 = c->p.nk[1], n3 = c->p.nk[2];
  auto iv = [&](int k, int d) { return d == 0 ? k / (n2 * n3) : d == 1 ? (k / n3) % n2 : k % n3; };
  std::vector<BdItem> A((size_t)nt * np), B((size_t)nt * np);
  for (int t = 0; t < nt; ++t) {
    const int tl = t % nc;
    for (long long lp = 0; lp < np; ++lp) {
      const long long p = pb + lp;
      const int k1 = c->pair_k1[1][p], k2 = c->pair_k2[1][p];
      int a = iv(k1, 0) - iv(k2, 0), b = iv(k1, 1) - iv(k2, 1), cc = iv(k1, 2) - iv(k2, 2);
      a = ((a % n1) + n1) % n1; b = ((b % n2) + n2) % n2; cc = ((cc % n3) + n3) % n3;
      const int q = (a * n2 + b) * n3 + cc;
      const long long pos = (lp * nc + tl) * vs;
      BdItem x;
      x.x_off = p * vs;
      x.y_off = pos;
      x.m_off = (long long)t * c->g_elems + c->g_off[c->rep[k2]];
      x.part = c->rep[k2];
      x.pad = 0;
      x.scale = z(1.0);
      A[(size_t)t * np + lp] = x;
      BdItem y;
      y.x_off = pos;
      y.y_off = pos;
      y.m_off = (long long)t * c->p_elems + c->p_off[c->rep[q]];
      y.part = c->rep[q];
      y.pad = 0;
      y.scale = z(1.0);
      B[(size_t)t * np + lp] = y;
    }
  }
  std::vector<GramUnit> units;
  std::vector<GramTile> tiles;
  P.unit_start.assign(nt + 1, 0);
  P.tile_start.assign(nt + 1, 0);
  long long base = 0;
  double work_t = 0;
  for (size_t b = 0; b < c->aob_off.size(); ++b) work_t += (double)c->aob_n[b] * c->aob_n[b] * c->naux * nao * Nk;
  const long long target = unit_target(work_t * nc);
  for (int t = 0; t < nt; ++t) {
    if (t % nc == 0) {
      if (t > 0) schedule_units(units, (size_t)base, 0);
      base = (long long)units.size();
    }
    P.unit_start[t] = units.size();
    P.tile_start[t] = tiles.size();
    const int tl = t % nc;
    for (size_t b = 0; b < c->aob_off.size(); ++b) {
      const int w = c->aob_w[b], nb = c->aob_n[b], st = c->aob_start[b];
      const long long p0 = std::max(pb, (long long)w * Nk), p1 = std::min(pe, (long long)(w + 1) * Nk);
      if (p1 <= p0) continue;
      const size_t from = units.size();
      add_gram_block(units, tiles, base, nb, (long long)t * c->g_elems + c->aob_off[b],
                     ((p0 - pb) * nc + tl) * vs + (long long)st * nao, p0 * vs + (long long)st * nao, nao, nao,
                     (int)(p1 - p0), (long long)c->naux * nao, target, c->herm);
      finalize_units(units, from, (long long)nc * vs, vs);
    }
  }
  schedule_units(units, (size_t)base, 0);
  P.unit_start[nt] = units.size();
  P.tile_start[nt] = tiles.size();
  P.max_units_chunk = 0;
  for (int t0 = 0; t0 < nt; t0 += nc) {
    const int t1 = std::min(nt, t0 + nc);
    P.max_units_chunk = std::max(P.max_units_chunk, P.unit_start[t1] - P.unit_start[t0]);
  }
  P.fl_A_t = P.fl_B_t = P.fl_G_t = 0;
  for (long long p = pb; p < pe; ++p) {
    const int k1 = c->pair_k1[1][p], k2 = c->pair_k2[1][p];
    int a = iv(k1, 0) - iv(k2, 0), b = iv(k1, 1) - iv(k2, 1), cc = iv(k1, 2) - iv(k2, 2);
    a = ((a % n1) + n1) % n1; b = ((b % n2) + n2) % n2; cc = ((cc % n3) + n3) % n3;
    P.fl_A_t += 8.0 * c->naux * nao * (double)c->part_ao[c->rep[k2]].elems;
    P.fl_B_t += 8.0 * nao * nao * (double)c->part_aux[c->rep[(a * n2 + b) * n3 + cc]].elems;
  }
  for (size_t b = 0; b < c->aob_n.size(); ++b) {
    const int w = c->aob_w[b];
    const long long npw = std::max(0LL, std::min(pe, (long long)(w + 1) * Nk) - std::max(pb, (long long)w * Nk));
    P.fl_G_t += 8.0 * npw * (double)c->naux * nao * gram_elems(c, c->aob_n[b]);
  }
  CKS(upload(c, P.d_A, A));
  CKS(upload(c, P.d_B, B));
  CKS(upload(c, P.d_units, units));
  CKS(upload(c, P.d_tiles, tiles));
  P.built = true;
  return SGW_OK;
}

template <typename Z>
static sgw_status self_energy_impl(sgw_ctx* c, const ContractionPlan& P, const Z* G, const Z* Pt, const Z* V,
                                   double2* out, cudaStream_t st, const char* tag) {
  const int nt = c->nt, nao = c->nao, naux = c->naux, nc = P.nc;
  const long long vs = vsize(c), np = P.items_per_t;
  const size_t inter = (size_t)np * nc * vs;
  CKS(ensure_workspace(c, (2 * inter + (size_t)P.max_units_chunk * 1024) * sizeof(Z)));
  Z* X1 = reinterpret_cast<Z*>(c->d_ws);
  Z* X2 = X1 + inter;
  Z* part = X2 + inter;
  GramGeom gg;
  gg.a_pair = (long long)nc * vs;
  gg.b_pair = vs;
  gg.a_row = nao;
  gg.b_row = nao;
  gg.k_outer_a = (long long)nao * nao;
  gg.k_outer_b = (long long)nao * nao;
  gg.k_inner = nao;
  gg.k_outer = naux;
  const std::string t_vg = std::string("sigma_vg") + tag, t_pvg = std::string("sigma_pvg") + tag,
                    t_gram = std::string("sigma_gram") + tag;
  for (int t0 = 0; t0 < nt; t0 += nc) {
    const int t1 = std::min(nt, t0 + nc);
    const long long ni = (long long)(t1 - t0) * np;
    const int ntc = t1 - t0;
    // X1[A][i][b] = sum_a V[A][i][a] G^{k2}(tau)[a][b]
    run(c, t_vg.c_str(), P.fl_A_t * ntc, 1, st, [&] {
      bdm(c, 0, geom(1, naux * nao, nao, 0, 0, 0, 0, nao), V, X1, G, P.d_A + (size_t)t0 * np, ni, st);
    });
    // X2[A'][(i,b)] = sum_A P^q(tau)[A][A'] X1[A][(i,b)]
    run(c, t_pvg.c_str(), P.fl_B_t * ntc, 1, st, [&] {
      bdm(c, 1, geom(1, naux, nao * nao, 1, 1, 0, 0, naux), X1, X2, Pt, P.d_B + (size_t)t0 * np, ni, st);
    });
    const long long u0 = P.unit_start[t0], u1 = P.unit_start[t1];
    const long long ti0 = P.tile_start[t0], ti1 = P.tile_start[t1];
    run(c, t_gram.c_str(), P.fl_G_t * ntc, 1, st, [&] { gram_partials(gg, X2, V, P.d_units + u0, (int)(u1 - u0), part, st); });
    run(c, "gram_reduce", 0.0, 1, st, [&] {
      gram_reduce(P.d_tiles + ti0, (int)(ti1 - ti0), part, out, z(-1.0 / c->Nk), 0, st);
    });
  }
  CKS(lower_from_upper(c, 0, out, st));
  return SGW_OK;
}

static sgw_status self_energy_range(sgw_ctx* c, const void* G_tau, const void* P_tau, void* Sigma_tau, long long pb,
                                    long long pe, sgw_stream stream) {
  CKS(need_built(c));
  if (!c->have_v[1]) return c->fail(SGW_ERR_STATE, "self-energy pairs of V not loaded");
  const long long np = (long long)c->nwedge * c->Nk;
  if (!G_tau || !P_tau || !Sigma_tau || pb < 0 || pe > np || pb > pe) return SGW_ERR_ARG;
  const bool whole = pb == 0 && pe == np;
  cudaStream_t st = S(stream);
  double2* out = static_cast<double2*>(Sigma_tau);
  if (!whole) CK(cudaMemsetAsync(out, 0, (size_t)c->nt * c->g_elems * sizeof(double2), st));
  if (pb == pe) return SGW_OK;
  ContractionPlan& P = whole ? c->plan_sigma : c->plan_sigma_part;
  if (!c->use_tc) CKS(build_sigma_plan(c, P, pb, pe));
  if (c->use_tc) {
    CKS(tc_self_energy(c, static_cast<const double2*>(G_tau), static_cast<const double2*>(P_tau), out, pb, pe, st));
  } else if (c->p.precision == SGW_MIXED_FP32) {
    const size_t gn = (size_t)c->nt * c->g_elems, pn = (size_t)c->nt * c->p_elems;
    CKS(ensure_g32(c, gn + pn));
    run(c, "convert", 0.0, 1, st, [&] { to_c64(static_cast<const double2*>(G_tau), c->d_g32, (long long)gn, st); });
    run(c, "convert", 0.0, 1, st, [&] { to_c64(static_cast<const double2*>(P_tau), c->d_g32 + gn, (long long)pn, st); });
    CKS(self_energy_impl<float2>(c, P, c->d_g32, c->d_g32 + gn, c->d_V32[1], out, st, "_f32"));
  } else {
    CKS(self_energy_impl<double2>(c, P, static_cast<const double2*>(G_tau), static_cast<const double2*>(P_tau),
                                  c->d_V[1], out, st, ""));
  }
  CK(cudaGetLastError());
  return SGW_OK;
}

extern "C" SGW_API sgw_status sgw_self_energy(sgw_ctx* c, const void* G_tau, const void* P_tau, void* Sigma_tau,
                                              sgw_stream stream) {
  if (!c) return SGW_ERR_ARG;
  return self_energy_range(c, G_tau, P_tau, Sigma_tau, 0, (long long)c->nwedge * c->Nk, stream);
}

extern "C" SGW_API sgw_status sgw_self_energy_pairs(sgw_ctx* c, const void* G_tau, const void* P_tau, void* Sigma_tau,
                                                    long long pair_begin, long long pair_end, sgw_stream stream) {
  if (!c) return SGW_ERR_ARG;
  return self_energy_range(c, G_tau, P_tau, Sigma_tau, pair_begin, pair_end, stream);
}

// ---------------------------------------------------------------------------
// a11: Hartree-Fock
// ---------------------------------------------------------------------------
static sgw_status density_matrix(sgw_ctx* c, const double2* G, double2* gamma, cudaStream_t st) {
  // gamma = -G(beta^-) = -sum_j beta_row[j] G(tau_j)
  run(c, "ft", 8.0 * c->nt * (double)c->g_elems, 1, st, [&] {
    series_map(c->d_beta_row, 1, c->nt, G, c->g_elems, gamma, c->g_elems, c->g_elems, z(-1.0), 0, st);
  });
  return SGW_OK;
}

// Exchange plan: wedge points are processed in groups whose Z = V gamma intermediates fit the
// workspace; one block multiply, one Gram launch and one reduction per group.
static sgw_status build_k_plan(sgw_ctx* c) {
  ContractionPlan& P = c->plan_k;
  if (P.built) return SGW_OK;
  const int Nk = c->Nk, nw = c->nwedge, nao = c->nao;
  const long long vs = vsize(c);
  const size_t budget = workspace_budget();
  int grp = (int)std::max<long long>(1, (long long)(budget * 0.5 / ((double)Nk * vs * sizeof(double2))));
  grp = std::min(grp, nw);
  P.nc = grp;  // wedge points per group
  std::vector<BdItem> A;
  std::vector<GramUnit> units;
  std::vector<GramTile> tiles;
  c->plan_k_wbeg.clear();
  c->plan_k_tbeg.clear();
  for (int w0 = 0; w0 < nw; w0 += grp) {
    const int w1 = std::min(nw, w0 + grp);
    c->plan_k_wbeg.push_back(units.size());
    c->plan_k_tbeg.push_back(tiles.size());
    for (int w = w0; w < w1; ++w)
      for (int k2 = 0; k2 < Nk; ++k2) {
        const long long p = (long long)w * Nk + k2;
        BdItem x;
        x.x_off = p * vs;
        x.y_off = (long long)((w - w0) * Nk + k2) * vs;
        x.m_off = c->g_off[c->rep[k2]];
        x.part = c->rep[k2];
        x.pad = 0;
        x.scale = z(1.0);
        A.push_back(x);
      }
    double work = 0;
    for (size_t b = 0; b < c->aob_off.size(); ++b)
      if (c->aob_w[b] >= w0 && c->aob_w[b] < w1) work += (double)c->aob_n[b] * c->aob_n[b] * c->naux * nao * Nk;
    const long long target = unit_target(work);
    const long long base = (long long)units.size();
    for (size_t b = 0; b < c->aob_off.size(); ++b) {
      const int w = c->aob_w[b];
      if (w < w0 || w >= w1) continue;
      const int nb = c->aob_n[b], st = c->aob_start[b];
      const size_t from = units.size();
      add_gram_block(units, tiles, base, nb, c->aob_off[b], (long long)(w - w0) * Nk * vs + (long long)st * nao,
                     (long long)w * Nk * vs + (long long)st * nao, nao, nao, Nk, (long long)c->naux * nao, target,
                     c->herm);
      finalize_units(units, from, vs, vs);
    }
    schedule_units(units, (size_t)base, 0);
  }
  c->plan_k_wbeg.push_back(units.size());
  c->plan_k_tbeg.push_back(tiles.size());
  P.max_units_chunk = 0;
  for (size_t g = 0; g + 1 < c->plan_k_wbeg.size(); ++g)
    P.max_units_chunk = std::max(P.max_units_chunk, c->plan_k_wbeg[g + 1] - c->plan_k_wbeg[g]);
  CKS(upload(c, P.d_A, A));
  CKS(upload(c, P.d_units, units));
  CKS(upload(c, P.d_tiles, tiles));
  // rho units: rho[A] = sum_k' sum_ab gamma^{k'}_ab conj(V^{k'k'}[A][a][b]), pairs (Gamma, k') of orientation 0
  ContractionPlan& R = c->plan_rho;
  std::vector<GramUnit> ru;
  std::vector<GramTile> rt;
  const int wG = c->rep[0];
  for (int A0 = 0; A0 < c->naux; A0 += 32) {
    GramTile t;
    t.tri = 0;
    t.out_off = A0;
    t.ld = 32;
    t.rows_m = 1;
    t.rows_n = std::min(32, c->naux - A0);
    t.unit_begin = (int)ru.size();
    t.unit_count = Nk;
    for (int kp = 0; kp < Nk; ++kp) {
      GramUnit u;
      u.rows_m = 1;
      u.rows_n = t.rows_n;
      u.r0 = 0;
      u.r1 = 1;
      u.a_off = (long long)c->rep[kp] * nao * nao;
      u.b_off = ((long long)wG * Nk + kp) * vs + (long long)A0 * nao * nao;
      u.slot = (int)ru.size();
      u.tri = 0;
      ru.push_back(u);
    }
    rt.push_back(t);
  }
  R.max_units_chunk = (long long)ru.size();
  CKS(upload(c, R.d_units, ru));
  CKS(upload(c, R.d_tiles, rt));
  R.built = true;
  P.built = true;
  return SGW_OK;
}

extern "C" SGW_API sgw_status sgw_hartree_fock(sgw_ctx* c, const void* G_tau, void* Sigma_hf, sgw_stream stream) {
  CKS(need_built(c));
  if (!c->have_v[0] || !c->have_v[1]) return c->fail(SGW_ERR_STATE, "V not loaded");
  if (!G_tau || !Sigma_hf) return SGW_ERR_ARG;
  CKS(build_k_plan(c));
  CKS(ensure_tables(c));
  cudaStream_t st = S(stream);
  const int Nk = c->Nk, nw = c->nwedge, nao = c->nao, naux = c->naux;
  const long long vs = vsize(c), mat = (long long)nao * nao;
  const size_t zbytes = (size_t)c->plan_k.nc * Nk * vs;
  const size_t need = zbytes + (size_t)c->plan_k.max_units_chunk * 1024 + c->plan_rho.max_units_chunk * 1024 +
                      c->g_elems + (size_t)nw * mat + naux + 16 + c->aob_off.size() * 2 + nw + 64;
  CKS(ensure_workspace(c, need * sizeof(double2)));
  double2* Zw = c->d_ws;
  double2* part = Zw + zbytes;
  double2* rpart = part + (size_t)c->plan_k.max_units_chunk * 1024;
  double2* gamma = rpart + c->plan_rho.max_units_chunk * 1024;
  double2* gdense = gamma + c->g_elems;
  double2* rho = gdense + (size_t)nw * mat;
  double2* out = static_cast<double2*>(Sigma_hf);
  density_matrix(c, static_cast<const double2*>(G_tau), gamma, st);
  // dense gamma per wedge point for the Hartree density
  {
    const size_t nb = c->aob_off.size();
    const long long* d_tab = c->d_hf_tab;
    const int* d_bn = reinterpret_cast<const int*>(d_tab + 2 * nb);
    run(c, "pack", 0.0, 1, st, [&] { fill_zero(gdense, (long long)nw * mat, st); });
    run(c, "pack", 0.0, 1, st, [&] {
      pack_blocks(gdense, mat, nao, d_tab, d_bn, d_tab + nb, (int)nb, gamma, 0, st);
    });
  }
  // rho[A]
  GramGeom rg;
  rg.a_pair = 0;
  rg.b_pair = 0;
  rg.a_row = 0;
  rg.b_row = mat;
  rg.k_outer_a = 0;
  rg.k_outer_b = 0;
  rg.k_inner = (int)mat;
  rg.k_outer = 1;
  run(c, "hf_j", 8.0 * Nk * (double)naux * mat, 1, st, [&] {
    gram_partials(rg, gdense, c->d_V[0], c->plan_rho.d_units, (int)c->plan_rho.max_units_chunk, rpart, st);
  });
  run(c, "gram_reduce", 0.0, 1, st, [&] { gram_reduce(c->plan_rho.d_tiles, (naux + 31) / 32, rpart, rho, z(1.0), 0, st); });
  // J^w_ij = (s/N_k) sum_A V^{k_w k_w}[A][i][j] rho[A]   (pair (Gamma, k_w) of orientation 0)
  {
    const long long* d_vw = c->d_hf_tab + 3 * c->aob_off.size();
    run(c, "hf_j", 8.0 * naux * (double)c->g_elems, 1, st, [&] {
      k_hartree<<<(unsigned)std::min<long long>(4096, (c->g_elems + 255) / 256), 256, 0, st>>>(
          c->d_V[0], rho, c->d_el_i, c->d_el_j, c->d_el_w, d_vw, c->g_elems, naux, nao,
          (double)c->p.spin_factor / Nk, out);
    });
  }
  // K^w = -(1/N_k) sum_k2 sum_A V(A) gamma^{k2} V(A)^dagger   (pairs (k_w, k2) of orientation 1)
  GramGeom gg;
  gg.a_pair = vs;
  gg.b_pair = vs;
  gg.a_row = nao;
  gg.b_row = nao;
  gg.k_outer_a = mat;
  gg.k_outer_b = mat;
  gg.k_inner = nao;
  gg.k_outer = naux;
  const int grp = c->plan_k.nc;
  for (size_t g = 0; g + 1 < c->plan_k_wbeg.size(); ++g) {
    const int w0 = (int)g * grp, w1 = std::min(nw, w0 + grp);
    double flz = 0, flg = 0;
    for (int w = w0; w < w1; ++w)
      for (int k2 = 0; k2 < Nk; ++k2) flz += 8.0 * naux * nao * (double)c->part_ao[c->rep[k2]].elems;
    for (size_t b = 0; b < c->aob_n.size(); ++b)
      if (c->aob_w[b] >= w0 && c->aob_w[b] < w1) flg += 8.0 * Nk * naux * nao * gram_elems(c, c->aob_n[b]);
    run(c, "hf_k", flz, 1, st, [&] {
      bdm(c, 0, geom(1, naux * nao, nao, 0, 0, 0, 0, nao), (const double2*)c->d_V[1], Zw, (const double2*)gamma,
          c->plan_k.d_A + (size_t)w0 * Nk, (long long)(w1 - w0) * Nk, st);
    });
    const long long u0 = c->plan_k_wbeg[g], u1 = c->plan_k_wbeg[g + 1];
    const long long t0 = c->plan_k_tbeg[g], t1 = c->plan_k_tbeg[g + 1];
    run(c, "hf_k", flg, 1, st, [&] {
      gram_partials(gg, Zw, c->d_V[1], c->plan_k.d_units + u0, (int)(u1 - u0), part, st);
    });
    run(c, "gram_reduce", 0.0, 1, st, [&] {
      gram_reduce(c->plan_k.d_tiles + t0, (int)(t1 - t0), part, out, z(-1.0 / Nk), 1, st);
    });
  }
  // K (and J, Hermitian for Hermitian gamma) was added on and above the diagonal only
  CKS(lower_from_upper(c, 2, out, st));
  CK(cudaGetLastError());
  return SGW_OK;
}

// ---------------------------------------------------------------------------
// a8-a10: Dyson with the chemical-potential search
// ---------------------------------------------------------------------------
// Dyson for the whole wedge at one chemical potential, or with the search of mu (bracketed
// Newton from the start point mu, or *mu_start_dev when given).  The search runs entirely on
// the device (no host round trip per trial): a fixed number of trial launches whose later
// members do nothing once the search has stopped.  The final mu is left in d_scalar[2].
static sgw_status dyson_device(sgw_ctx* c, const double2* Sigma_tau, const double2* Sigma_hf, double mu,
                               int search_mu, double2* G_tau, cudaStream_t st,
                               const double* mu_start_dev = nullptr) {
  CKS(ensure_tables(c));
  const long long ge = c->g_elems;
  const int nwf = c->nwf;
  const int maxn = c->max_ao_block;
  const size_t scratch = maxn > 90 ? (size_t)304 * maxn * maxn : 0;
  const size_t need = (size_t)2 * nwf * ge + ge + scratch + c->n_dy_items + 64;
  CKS(ensure_workspace(c, need * sizeof(double2)));
  double2* Sw = c->d_ws;
  double2* Gw = Sw + (size_t)nwf * ge;
  double2* F = Gw + (size_t)nwf * ge;
  double2* scr = F + ge;
  double2* tpart = scr + scratch;
  double fli = 0;
  for (size_t b = 0; b < c->aob_n.size(); ++b) fli += 8.0 * nwf * std::pow((double)c->aob_n[b], 3);
  run(c, "ft", 8.0 * nwf * (double)c->nt * ge, 1, st, [&] {
    series_map(c->d_TF, nwf, c->nt, Sigma_tau, ge, Sw, ge, ge, z(1.0), 0, st);
  });
  CK(cudaMemcpyAsync(F, c->d_H0, ge * sizeof(double2), cudaMemcpyDeviceToDevice, st));
  run(c, "axpby", 0.0, 1, st, [&] { axpby(F, Sigma_hf, ge, 1.0, 1.0, st); });
  double* s = c->d_scalar;
  const double* mu_dev = nullptr;
  if (search_mu) {
    run(c, "mu_search", 0.0, 1, st, [&] { mu_start(s, mu, mu_start_dev, -20.0, 20.0, st); });
    // a trial inverts every block (n^3) and forms G S (n^3) for the slope; the flops of the
    // trials that ran are added from the device's trial count when the profile is read
    c->dy_trial_flops = 2.0 * fli;
    for (int it = 0; it < 64; ++it) {
      run(c, "dyson_invert", 0.0, 1, st, [&] {
        invert_plan(INV_DYSON_TRACE, c->dy_plan, Sw, c->d_S, F, c->d_nu_f, 0.0, s + 2, s + 3, nullptr, tpart, scr,
                    c->d_status, st);
      });
      run(c, "mu_search", 0.0, 1, st, [&] { mu_update(s, tpart, c->n_dy_items, c->p.n_elec, 1e-11, st); });
    }
    mu_dev = s + 2;
  }
  run(c, "dyson_invert", fli, 1, st, [&] {
    invert_plan(INV_DYSON_STORE, c->dy_plan, Sw, c->d_S, F, c->d_nu_f, mu, mu_dev, nullptr, Gw, nullptr, scr,
                c->d_status, st);
  });
  run(c, "ft", 8.0 * nwf * (double)c->nt * ge, 1, st, [&] {
    series_map(c->d_TFbar, c->nt, nwf, Gw, ge, G_tau, ge, ge, z(1.0), 0, st);
  });
  CKS(hermitian_g(c, G_tau, st));
  CK(cudaGetLastError());
  return SGW_OK;
}

extern "C" SGW_API sgw_status sgw_dyson(sgw_ctx* c, const void* Sigma_tau, const void* Sigma_hf, double* mu_inout,
                                        int search_mu, void* G_tau, sgw_stream stream) {
  CKS(need_built(c));
  if (!c->have_one_body) return c->fail(SGW_ERR_STATE, "one-body inputs not loaded");
  if (!Sigma_tau || !Sigma_hf || !mu_inout || !G_tau) return SGW_ERR_ARG;
  cudaStream_t st = S(stream);
  CKS(dyson_device(c, static_cast<const double2*>(Sigma_tau), static_cast<const double2*>(Sigma_hf), *mu_inout,
                   search_mu, static_cast<double2*>(G_tau), st));
  if (search_mu) {
    double sc[5] = {0, 0, 0, 0, 0};  // lo, hi, mu, done, N of the last trial
    CK(cudaMemcpyAsync(sc, c->d_scalar, sizeof(sc), cudaMemcpyDeviceToHost, st));
    CKS(sgw_sync(c, stream));
    *mu_inout = sc[2];
    if (sc[3] == 0.0)
      return c->fail(SGW_ERR_NOCONV, "mu search: |N - n_elec| = " + std::to_string(std::fabs(sc[4] - c->p.n_elec)) +
                                         " after 64 trials (bracket [" + std::to_string(sc[0]) + ", " +
                                         std::to_string(sc[1]) + "]); G was built at the last mu");
  }
  return SGW_OK;
}

// ---------------------------------------------------------------------------
// a12: energy
// ---------------------------------------------------------------------------
extern "C" SGW_API sgw_status sgw_energy(sgw_ctx* c, const void* G_tau, const void* Sigma_hf, const void* Sigma_tau,
                                         double* e_out, sgw_stream stream) {
  CKS(need_built(c));
  if (!G_tau || !Sigma_hf || !Sigma_tau || !e_out) return SGW_ERR_ARG;
  cudaStream_t st = S(stream);
  const long long ge = c->g_elems;
  const int nt = c->nt;
  const double s = c->p.spin_factor, Nk = c->Nk;
  const size_t nb = c->aob_off.size();
  const size_t ntr = nb * (size_t)(2 + nt);
  const size_t need = ge + (size_t)2 * nt * ge + ntr + ntr * sizeof(TrItem) / 16 + 64;
  CKS(ensure_workspace(c, need * sizeof(double2)));
  double2* gamma = c->d_ws;
  double2* Gg = gamma + ge;
  double2* Sg = Gg + (size_t)nt * ge;
  double2* part = Sg + (size_t)nt * ge;
  TrItem* d_items = reinterpret_cast<TrItem*>(part + ntr + 8);
  density_matrix(c, static_cast<const double2*>(G_tau), gamma, st);
  run(c, "ft", 8.0 * nt * (double)nt * ge, 1, st, [&] {
    series_map(c->d_gl_interp, nt, nt, static_cast<const double2*>(G_tau), ge, Gg, ge, ge, z(1.0), 0, st);
  });
  run(c, "ft", 8.0 * nt * (double)nt * ge, 1, st, [&] {
    series_map(c->d_gl_interp, nt, nt, static_cast<const double2*>(Sigma_tau), ge, Sg, ge, ge, z(1.0), 0, st);
  });
  double2* d_res = reinterpret_cast<double2*>(c->d_scalar);
  double out[3][2];
  for (int term = 0; term < 3; ++term) {
    std::vector<TrItem> items;
    for (size_t b = 0; b < nb; ++b) {
      const double star = c->star[c->aob_w[b]];
      if (term < 2) {
        TrItem t;
        t.x_off = c->aob_off[b];
        t.y_off = c->aob_off[b];
        t.n = c->aob_n[b];
        t.pad = 0;
        t.w = z(term == 0 ? s / Nk * star : s / (2 * Nk) * star);
        items.push_back(t);
      } else {
        for (int g = 0; g < nt; ++g) {
          TrItem t;
          t.x_off = (long long)g * ge + c->aob_off[b];
          t.y_off = (long long)(nt - 1 - g) * ge + c->aob_off[b];
          t.n = c->aob_n[b];
          t.pad = 0;
          t.w = z(-(s / (2 * Nk)) * 0.5 * c->p.beta * c->gl_w[g] * star);
          items.push_back(t);
        }
      }
    }
    CK(cudaMemcpyAsync(d_items, items.data(), items.size() * sizeof(TrItem), cudaMemcpyHostToDevice, st));
    const double2* X = term == 2 ? Gg : gamma;
    const double2* Y = term == 0 ? c->d_H0 : term == 1 ? static_cast<const double2*>(Sigma_hf) : Sg;
    run(c, "trace", 0.0, 2, st, [&] { trace_products(d_items, (int)items.size(), X, Y, part, d_res, st); });
    double2 h;
    CK(cudaMemcpyAsync(&h, d_res, sizeof(double2), cudaMemcpyDeviceToHost, st));
    CK(cudaStreamSynchronize(st));
    out[term][0] = h.x;
    out[term][1] = h.y;
  }
  e_out[0] = out[0][0] + out[1][0] + out[2][0];
  e_out[1] = out[0][0];
  e_out[2] = out[1][0];
  e_out[3] = out[2][0];
  e_out[4] = out[0][1] + out[1][1] + out[2][1];
  return SGW_OK;
}

// ---------------------------------------------------------------------------
// a2..a12: iterate
// ---------------------------------------------------------------------------
// One pass, enqueued on `st` only (capturable): P0 -> P -> Sigma~, Sigma_HF -> damping ->
// max |Delta Sigma| -> Dyson with the device-side mu search; the scalars the host needs
// (mu, N, max |Delta Sigma|) are copied into pinned host memory at the end of the pass.
static sgw_status iteration_body(sgw_ctx* c, double damping, double2* G, double2* Sig, double2* Hf, cudaStream_t st) {
  const long long ge = c->g_elems;
  const int nt = c->nt;
  sgw_stream ss = reinterpret_cast<sgw_stream>(st);
  CKS(sgw_polarization(c, G, c->d_it_P0, ss));
  CKS(sgw_screened_interaction(c, c->d_it_P0, c->d_it_P, ss));
  CKS(sgw_self_energy(c, G, c->d_it_P, c->d_it_S, ss));
  CKS(sgw_hartree_fock(c, G, c->d_it_H, ss));
  // Sigma <- (1 - a) Sigma_old + a Sigma_new, and max |Sigma_damped - Sigma_old|
  run(c, "axpby", 0.0, 1, st, [&] { axpby(c->d_it_S, Sig, (long long)nt * ge, damping, 1.0 - damping, st); });
  run(c, "axpby", 0.0, 1, st, [&] { axpby(c->d_it_H, Hf, ge, damping, 1.0 - damping, st); });
  run(c, "reduce", 0.0, 1, st, [&] { max_abs_diff(c->d_it_S, Sig, (long long)nt * ge, c->d_maxbits, st); });
  run(c, "reduce", 0.0, 1, st, [&] { max_abs_diff(c->d_it_H, Hf, ge, c->d_maxbits + 1, st); });
  CK(cudaMemcpyAsync(Sig, c->d_it_S, (size_t)nt * ge * sizeof(double2), cudaMemcpyDeviceToDevice, st));
  CK(cudaMemcpyAsync(Hf, c->d_it_H, (size_t)ge * sizeof(double2), cudaMemcpyDeviceToDevice, st));
  // the search starts at the mu the host put in h_pinned[12] before this pass (read when the pass runs)
  CK(cudaMemcpyAsync(c->d_scalar + 6, c->h_pinned + 12, sizeof(double), cudaMemcpyHostToDevice, st));
  CKS(dyson_device(c, Sig, Hf, 0.0, 1, G, st, c->d_scalar + 6));
  CK(cudaMemcpyAsync(c->h_pinned, c->d_scalar, 8 * sizeof(double), cudaMemcpyDeviceToHost, st));
  CK(cudaMemcpyAsync(c->h_pinned + 8, c->d_maxbits, 2 * sizeof(unsigned long long), cudaMemcpyDeviceToHost, st));
  return SGW_OK;
}

static bool graphs_enabled() {
  const char* e = std::getenv("SGW_GRAPH");
  return !(e && e[0] == '0');
}

extern "C" SGW_API sgw_status sgw_iterate(sgw_ctx* c, int max_iter, double damping, double tol, void* G_tau,
                                          void* Sigma_tau, void* Sigma_hf, double* mu, sgw_iter_stats* stats,
                                          sgw_stream stream) {
  CKS(need_built(c));
  if (!G_tau || !Sigma_tau || !Sigma_hf || !mu || max_iter < 1 || !(damping > 0) || damping > 1)
    return SGW_ERR_ARG;
  if (!c->have_one_body || !c->have_v[0] || !c->have_v[1]) return c->fail(SGW_ERR_STATE, "inputs not loaded");
  cudaStream_t st = S(stream);
  const long long ge = c->g_elems, pe = c->p_elems;
  const int nt = c->nt;
  if (!c->d_it_P0) {
    if (cudaMalloc(&c->d_it_P0, (size_t)nt * pe * sizeof(double2)) != cudaSuccess ||
        cudaMalloc(&c->d_it_P, (size_t)nt * pe * sizeof(double2)) != cudaSuccess ||
        cudaMalloc(&c->d_it_S, (size_t)nt * ge * sizeof(double2)) != cudaSuccess ||
        cudaMalloc(&c->d_it_H, (size_t)ge * sizeof(double2)) != cudaSuccess ||
        cudaMallocHost(&c->h_pinned, 16 * sizeof(double)) != cudaSuccess)
      return c->fail(SGW_ERR_OOM, "iteration buffers");
  }
  double2* G = static_cast<double2*>(G_tau);
  double2* Sig = static_cast<double2*>(Sigma_tau);
  double2* Hf = static_cast<double2*>(Sigma_hf);
  // a graph needs a capturable (non-legacy) stream and no per-kernel event timing
  const bool graph = graphs_enabled() && st != nullptr && !c->prof_on && c->it_warm;
  if (graph && (c->it_exec == nullptr || c->it_key[0] != G || c->it_key[1] != Sig || c->it_key[2] != Hf ||
                c->it_damping != damping || c->it_gen != c->ws_gen)) {
    if (c->it_exec) cudaGraphExecDestroy(c->it_exec);
    if (c->it_graph) cudaGraphDestroy(c->it_graph);
    c->it_exec = nullptr;
    c->it_graph = nullptr;
    CK(cudaStreamBeginCapture(st, cudaStreamCaptureModeThreadLocal));
    sgw_status sb = iteration_body(c, damping, G, Sig, Hf, st);
    cudaGraph_t g = nullptr;
    cudaError_t ec = cudaStreamEndCapture(st, &g);
    if (sb != SGW_OK) {
      if (g) cudaGraphDestroy(g);
      return sb;
    }
    if (ec != cudaSuccess) return c->fail(SGW_ERR_CUDA, std::string("graph capture: ") + cudaGetErrorString(ec));
    c->it_graph = g;
    CK(cudaGraphInstantiate(&c->it_exec, g, 0));
    c->it_key[0] = G;
    c->it_key[1] = Sig;
    c->it_key[2] = Hf;
    c->it_damping = damping;
    c->it_gen = c->ws_gen;
  }
  double dmax = 0.0;
  int it = 0;
  for (it = 0; it < max_iter; ++it) {
    c->h_pinned[12] = *mu;  // start of this pass's mu search (the stream is idle here)
    if (graph) {
      CK(cudaGraphLaunch(c->it_exec, st));
    } else {
      CKS(iteration_body(c, damping, G, Sig, Hf, st));
    }
    CK(cudaStreamSynchronize(st));
    c->it_warm = 1;
    double d1, d2;
    std::memcpy(&d1, c->h_pinned + 8, 8);
    std::memcpy(&d2, c->h_pinned + 9, 8);
    dmax = std::max(d1, d2);
    *mu = c->h_pinned[2];
    if (c->h_pinned[3] == 0.0) {  // the pass's mu search stopped without meeting its tolerance
      CKS(sgw_sync(c, stream));
      return c->fail(SGW_ERR_NOCONV, "mu search of pass " + std::to_string(it + 1) + ": |N - n_elec| = " +
                                         std::to_string(std::fabs(c->h_pinned[4] - c->p.n_elec)) + " after 64 trials");
    }
    if (dmax < tol) { ++it; break; }
  }
  CKS(sgw_sync(c, stream));
  if (stats) {
    stats->iterations = it;
    stats->mu = *mu;
    stats->max_dsigma = dmax;
    stats->n_elec = c->h_pinned[4];
    double e[5];
    CKS(sgw_energy(c, G_tau, Sigma_hf, Sigma_tau, e, stream));
    for (int i = 0; i < 4; ++i) stats->energy[i] = e[i];
    stats->energy_imag = e[4];
  }
  return SGW_OK;
}

// ---------------------------------------------------------------------------
// unfolding to the AO basis over the whole zone
// ---------------------------------------------------------------------------
extern "C" SGW_API sgw_status sgw_unfold(sgw_ctx* c, int which, int nt, const void* packed, void* ao_full,
                                         sgw_stream stream) {
  CKS(need_built(c));
  if ((which != 0 && which != 1) || nt < 1 || !packed || !ao_full) return SGW_ERR_ARG;
  cudaStream_t st = S(stream);
  const int n = which == 0 ? c->nao : c->naux, Nk = c->Nk;
  const long long mat = (long long)n * n, elems = which == 0 ? c->g_elems : c->p_elems;
  const auto& boff = which == 0 ? c->aob_off : c->auxb_off;
  const auto& bnn = which == 0 ? c->aob_n : c->auxb_n;
  const auto& bw = which == 0 ? c->aob_w : c->auxb_w;
  const auto& bst = which == 0 ? c->aob_start : c->auxb_start;
  // dense block matrices per (k, t), then X = U Y U^dagger
  std::vector<long long> bdo, bpo;
  std::vector<int> bn;
  for (int k = 0; k < Nk; ++k)
    for (int t = 0; t < nt; ++t)
      for (size_t b = 0; b < boff.size(); ++b) {
        if (bw[b] != c->rep[k]) continue;
        bdo.push_back(((long long)k * nt + t) * mat + (long long)bst[b] * n + bst[b]);
        bpo.push_back((long long)t * elems + boff[b]);
        bn.push_back(bnn[b]);
      }
  const size_t need = (size_t)Nk * nt * mat + (bdo.size() * 2 + bn.size()) + (size_t)Nk * nt * 3 + 64;
  CKS(ensure_workspace(c, need * sizeof(double2)));
  double2* Y = c->d_ws;
  long long* d_bdo = reinterpret_cast<long long*>(Y + (size_t)Nk * nt * mat);
  long long* d_bpo = d_bdo + bdo.size();
  int* d_bn = reinterpret_cast<int*>(d_bpo + bpo.size());
  // item table on a 16-byte boundary after the integer table
  const uintptr_t tail = reinterpret_cast<uintptr_t>(d_bn + bn.size());
  BdItem* d_items = reinterpret_cast<BdItem*>((tail + 15) & ~static_cast<uintptr_t>(15));
  CK(cudaMemcpyAsync(d_bdo, bdo.data(), bdo.size() * 8, cudaMemcpyHostToDevice, st));
  CK(cudaMemcpyAsync(d_bpo, bpo.data(), bpo.size() * 8, cudaMemcpyHostToDevice, st));
  CK(cudaMemcpyAsync(d_bn, bn.data(), bn.size() * 4, cudaMemcpyHostToDevice, st));
  run(c, "pack", 0.0, 1, st, [&] { fill_zero(Y, (long long)Nk * nt * mat, st); });
  run(c, "pack", 0.0, 1, st, [&] {
    pack_blocks(Y, mat, n, d_bdo, d_bn, d_bpo, (int)bn.size(), const_cast<double2*>(static_cast<const double2*>(packed)),
                0, st);
  });
  std::vector<BdItem> items((size_t)Nk * nt);
  for (int k = 0; k < Nk; ++k)
    for (int t = 0; t < nt; ++t) {
      BdItem& x = items[(size_t)k * nt + t];
      x.x_off = ((long long)k * nt + t) * mat;
      x.y_off = x.x_off;
      x.m_off = (long long)k * mat;
      x.part = which;
      x.pad = 0;
      x.scale = z(1.0);
    }
  CK(cudaMemcpyAsync(d_items, items.data(), items.size() * sizeof(BdItem), cudaMemcpyHostToDevice, st));
  const int W = std::max(c->nao, c->naux);
  const double2* U = which == 0 ? c->d_Uao : c->d_Uaux;
  double2* out = static_cast<double2*>(ao_full);
  const double flu = 8.0 * items.size() * (double)n * n * n;
  run(c, "unfold", flu, 1, st, [&] {
    bd_mult(geom(1, n, n, 1, 0, 0, 0, W), Y, out, U, d_items, (long long)items.size(), c->d_full_start,
            c->d_full_size, c->d_full_doff, st);
  });
  run(c, "unfold", flu, 1, st, [&] {
    bd_mult(geom(1, n, n, 0, 1, 1, 0, W), out, Y, U, d_items, (long long)items.size(), c->d_full_start,
            c->d_full_size, c->d_full_doff, st);
  });
  CK(cudaMemcpyAsync(out, Y, (size_t)Nk * nt * mat * sizeof(double2), cudaMemcpyDeviceToDevice, st));
  CK(cudaStreamSynchronize(st));
  return SGW_OK;
}

// ---------------------------------------------------------------------------
// instrumentation
// ---------------------------------------------------------------------------
// running count of evaluated mu-search trials (d_scalar[16]); synchronises the device
static double trials_done(sgw_ctx* c) {
  double v = 0.0;
  if (c->d_scalar && cudaDeviceSynchronize() == cudaSuccess && cudaMemcpy(&v, c->d_scalar + 16, sizeof(double), cudaMemcpyDeviceToHost) != cudaSuccess) v = 0.0;
  return v;
}

extern "C" SGW_API sgw_status sgw_set_wait_limit(sgw_ctx* c, unsigned long long ns) {
  if (!c) return SGW_ERR_ARG;
  c->tc_wait_ns = ns;
  return SGW_OK;
}

extern "C" SGW_API sgw_status sgw_profile_enable(sgw_ctx* c, int on) {
  if (!c) return SGW_ERR_ARG;
  if (on && !c->prof_on) c->prof_trials_seen = trials_done(c);
  c->prof_on = on != 0;
  return SGW_OK;
}

extern "C" SGW_API sgw_status sgw_profile_read(sgw_ctx* c, int max_entries, char* names, double* ms, double* gflop,
                                               long long* launches, int* n_out, int reset) {
  if (!c || !n_out) return SGW_ERR_ARG;
  for (auto& e : c->prof_pending) {
    cudaEventSynchronize(e.b);
    float t = 0.f;
    cudaEventElapsedTime(&t, e.a, e.b);
    c->prof_ms[e.id] += t;
    cudaEventDestroy(e.a);
    cudaEventDestroy(e.b);
  }
  c->prof_pending.clear();
  if (c->dy_trial_flops > 0.0) {
    const double t = trials_done(c);
    for (size_t i = 0; i < c->prof_names.size(); ++i)
      if (c->prof_names[i] == "dyson_invert") c->prof_flops[i] += (t - c->prof_trials_seen) * c->dy_trial_flops;
    c->prof_trials_seen = t;
  }
  const int n = (int)c->prof_names.size();
  *n_out = n;
  for (int i = 0; i < n && i < max_entries; ++i) {
    if (names) {
      std::strncpy(names + 48 * i, c->prof_names[i].c_str(), 47);
      names[48 * i + 47] = 0;
    }
    if (ms) ms[i] = c->prof_ms[i];
    if (gflop) gflop[i] = c->prof_flops[i] * 1e-9;
    if (launches) launches[i] = c->prof_launch[i];
  }
  if (reset) {
    std::fill(c->prof_ms.begin(), c->prof_ms.end(), 0.0);
    std::fill(c->prof_flops.begin(), c->prof_flops.end(), 0.0);
    std::fill(c->prof_launch.begin(), c->prof_launch.end(), 0LL);
  }
  return SGW_OK;
}

// ---------------------------------------------------------------------------
// host-only set-up queries (no device needed)
// ---------------------------------------------------------------------------
static bool params_ok(const sgw_params* p) {
  return p && p->nk[0] >= 1 && p->nk[1] >= 1 && p->nk[2] >= 1 && p->nao >= 1 && p->naux >= 1 && p->ntau >= 2 &&
         p->nw_f >= p->ntau && p->nw_b >= p->ntau && p->mats_f && p->mats_b && p->beta > 0;
}

static void host_ctx(const sgw_params* p, sgw_ctx& c) {
  c.p = *p;
  c.mats_f.assign(p->mats_f, p->mats_f + p->nw_f);
  c.mats_b.assign(p->mats_b, p->mats_b + p->nw_b);
  c.Nk = p->nk[0] * p->nk[1] * p->nk[2];
  c.nao = p->nao;
  c.naux = p->naux;
  c.nt = p->ntau;
  c.nwf = p->nw_f;
  c.nwb = p->nw_b;
}

extern "C" SGW_API sgw_status sgw_host_grid(const sgw_params* p, double* tau, double* TF, double* TFbar, double* TB,
                                            double* TBbar) {
  if (!params_ok(p)) return SGW_ERR_ARG;
  sgw_ctx c;
  host_ctx(p, c);
  sgw_status s = build_grid(&c);
  if (s != SGW_OK) return s;
  auto put = [](double* dst, const std::vector<cplx>& v) {
    if (!dst) return;
    for (size_t i = 0; i < v.size(); ++i) { dst[2 * i] = v[i].real(); dst[2 * i + 1] = v[i].imag(); }
  };
  if (tau) std::copy(c.tau.begin(), c.tau.end(), tau);
  put(TF, c.TF);
  put(TFbar, c.TFbar);
  put(TB, c.TB);
  put(TBbar, c.TBbar);
  return SGW_OK;
}

extern "C" SGW_API sgw_status sgw_host_irrep_dims(const sgw_params* p, const sgw_structure* st, int* nwedge,
                                                  int* ao_dims, int* aux_dims) {
  if (!params_ok(p) || !st || !nwedge) return SGW_ERR_ARG;
  sgw_ctx c;
  host_ctx(p, c);
  sgw_status s = build_symmetry(&c, st);
  if (s != SGW_OK) return s;
  *nwedge = c.nwedge;
  for (int w = 0; w < c.nwedge; ++w) {
    for (int fam = 0; fam < 2; ++fam) {
      int* out = fam == 0 ? ao_dims : aux_dims;
      if (!out) continue;
      const Partition& P = fam == 0 ? c.part_ao[w] : c.part_aux[w];
      int* row = out + (size_t)w * ((fam == 0 ? c.nao : c.naux) + 1);
      int i = 0;
      for (int d : P.dims) row[i++] = d;
      row[i] = 0;
    }
  }
  return SGW_OK;
}

extern "C" SGW_API sgw_status sgw_host_partner_basis(const sgw_params* p, const sgw_structure* st, int family,
                                                     int* nwedge, double* U) {
  if (!params_ok(p) || !st || !nwedge || (family != 0 && family != 1)) return SGW_ERR_ARG;
  sgw_ctx c;
  host_ctx(p, c);
  c.want_partner = true;
  sgw_status s = build_symmetry(&c, st);
  if (s != SGW_OK) return s;
  *nwedge = c.nwedge;
  if (U) {
    const size_t nn = (size_t)(family == 0 ? c.nao : c.naux) * (family == 0 ? c.nao : c.naux);
    for (int w = 0; w < c.nwedge; ++w) {
      const auto& X = c.partner_U[family][w];
      for (size_t e = 0; e < nn; ++e) {
        U[2 * ((size_t)w * nn + e)] = X[e].real();
        U[2 * ((size_t)w * nn + e) + 1] = X[e].imag();
      }
    }
  }
  return SGW_OK;
}

extern "C" SGW_API sgw_status sgw_host_symmetry(const sgw_params* p, const sgw_structure* st, int* nwedge, int* rep,
                                                int* ao_blocks, int* aux_blocks) {
  if (!params_ok(p) || !st || !nwedge) return SGW_ERR_ARG;
  sgw_ctx c;
  host_ctx(p, c);
  sgw_status s = build_symmetry(&c, st);
  if (s != SGW_OK) return s;
  *nwedge = c.nwedge;
  if (rep) std::copy(c.rep.begin(), c.rep.end(), rep);
  for (int w = 0; w < c.nwedge; ++w) {
    if (ao_blocks) {
      int* row = ao_blocks + (size_t)w * (c.nao + 1);
      int i = 0;
      for (int sz : c.part_ao[w].sizes) row[i++] = sz;
      row[i] = 0;
    }
    if (aux_blocks) {
      int* row = aux_blocks + (size_t)w * (c.naux + 1);
      int i = 0;
      for (int sz : c.part_aux[w].sizes) row[i++] = sz;
      row[i] = 0;
    }
  }
  return SGW_OK;
}
