// Set-up of the sgw context: tau grid and Matsubara transforms, and the space-group
// analysis of Algorithm 1 (orbital representation, projective representation,
// Dirac characters, simultaneous diagonalisation, stars).  Runs once per context.
#include <algorithm>
#include <array>
#include <cmath>
#include <cstring>
#include <map>
#include <numeric>
#include <random>
#include <set>

#include "sgw_internal.h"

namespace sgw {

static const double kPi = 3.14159265358979323846;

// ---------------------------------------------------------------------------
// small dense complex helpers (row-major)
// ---------------------------------------------------------------------------
static void gauss_legendre(int n, std::vector<double>& x, std::vector<double>& w) {
  // Newton iteration on P_n, starting from the Chebyshev-like guesses.
  x.assign(n, 0.0);
  w.assign(n, 0.0);
  for (int i = 0; i < n; ++i) {
    double z = std::cos(kPi * (i + 0.75) / (n + 0.5));
    for (int it = 0; it < 100; ++it) {
      double p0 = 1.0, p1 = 0.0;
      for (int j = 1; j <= n; ++j) {
        const double p2 = p1;
        p1 = p0;
        p0 = ((2.0 * j - 1.0) * z * p1 - (j - 1.0) * p2) / j;
      }
      const double dp = n * (z * p0 - p1) / (z * z - 1.0);
      const double dz = p0 / dp;
      z -= dz;
      if (std::fabs(dz) < 1e-16) {
        double q0 = 1.0, q1 = 0.0;
        for (int j = 1; j <= n; ++j) {
          const double q2 = q1;
          q1 = q0;
          q0 = ((2.0 * j - 1.0) * z * q1 - (j - 1.0) * q2) / j;
        }
        const double dq = n * (z * q0 - q1) / (z * z - 1.0);
        x[i] = -z;
        w[i] = 2.0 / ((1.0 - z * z) * dq * dq);
        break;
      }
    }
  }
  std::vector<int> idx(n);
  std::iota(idx.begin(), idx.end(), 0);
  std::sort(idx.begin(), idx.end(), [&](int a, int b) { return x[a] < x[b]; });
  std::vector<double> xs(n), ws(n);
  for (int i = 0; i < n; ++i) { xs[i] = x[idx[i]]; ws[i] = w[idx[i]]; }
  x = xs;
  w = ws;
}

// int_{-1}^{1} e^{i a x} T_l(x) dx for l < n, by integration by parts (exact, |a| >= (n-1)^2)
// or composite 16-point Gauss-Legendre (refined until stable).
static void fourier_cheb(double a, int n, double zeta, std::vector<cplx>& out) {
  out.assign(n, cplx(0, 0));
  if (std::fabs(a) >= std::max(1.0, (n - 1.0) * (n - 1.0))) {
    const cplx ia(0.0, a);
    for (int l = 0; l < n; ++l) {
      double deriv = 1.0;  // T_l^{(k)}(1)
      cplx pw = ia, acc(0, 0);
      for (int k = 0; k <= l; ++k) {
        const double sgn_k = (k & 1) ? -1.0 : 1.0;
        const double sgn_lk = ((l + k) & 1) ? -1.0 : 1.0;
        acc += sgn_k * deriv * (zeta - sgn_lk) / pw;
        deriv *= (double)(l * l - k * k) / (2.0 * k + 1.0);
        pw *= ia;
      }
      out[l] = acc;  // = e^{-ia} * int e^{ia(1+x)} T_l dx, see caller
    }
    return;
  }
  static std::vector<double> gx, gw;
  if (gx.empty()) gauss_legendre(16, gx, gw);
  long long panels = (long long)std::ceil((std::fabs(a) + n) / kPi) + 2;
  std::vector<cplx> prev;
  // The first rule already resolves the integrand; refine until two rules agree to the
  // rounding floor of the sums (the integrals are O(1)), at most a few doublings.
  for (int rep = 0; rep < 8; ++rep) {
    std::vector<cplx> cur(n, cplx(0, 0));
    const double h = 2.0 / panels;
    for (long long p = 0; p < panels; ++p) {
      const double mid = -1.0 + (p + 0.5) * h;
      for (int q = 0; q < 16; ++q) {
        const double x = mid + 0.5 * h * gx[q];
        const double wq = 0.5 * h * gw[q];
        const cplx ph = std::exp(cplx(0.0, a * (1.0 + x))) * wq;
        const double th = std::acos(std::max(-1.0, std::min(1.0, x)));
        for (int l = 0; l < n; ++l) cur[l] += ph * std::cos(l * th);
      }
    }
    if (!prev.empty()) {
      double d = 0;
      for (int l = 0; l < n; ++l) d = std::max(d, std::abs(cur[l] - prev[l]));
      if (d <= 2e-14) { out = cur; return; }
    }
    prev = cur;
    panels *= 2;
  }
  out = prev;
}

// Pseudo-inverse of a full-column-rank m x n complex matrix via Householder QR.
static std::vector<cplx> pinv_qr(const std::vector<cplx>& T, int m, int n) {
  std::vector<cplx> R(T), Qh((size_t)m * m, cplx(0, 0));
  for (int i = 0; i < m; ++i) Qh[(size_t)i * m + i] = 1.0;
  for (int k = 0; k < n; ++k) {
    double nx = 0;
    for (int i = k; i < m; ++i) nx += std::norm(R[(size_t)i * n + k]);
    nx = std::sqrt(nx);
    if (nx == 0) continue;
    const cplx x0 = R[(size_t)k * n + k];
    const cplx ph = std::abs(x0) > 0 ? x0 / std::abs(x0) : cplx(1, 0);
    const cplx alpha = -ph * nx;
    std::vector<cplx> v(m - k);
    for (int i = k; i < m; ++i) v[i - k] = R[(size_t)i * n + k];
    v[0] -= alpha;
    double nv = 0;
    for (auto& z : v) nv += std::norm(z);
    nv = std::sqrt(nv);
    if (nv == 0) continue;
    for (auto& z : v) z /= nv;
    for (int j = k; j < n; ++j) {  // R <- (I - 2 v v^H) R
      cplx s(0, 0);
      for (int i = k; i < m; ++i) s += std::conj(v[i - k]) * R[(size_t)i * n + j];
      for (int i = k; i < m; ++i) R[(size_t)i * n + j] -= 2.0 * v[i - k] * s;
    }
    for (int j = 0; j < m; ++j) {  // Qh <- (I - 2 v v^H) Qh
      cplx s(0, 0);
      for (int i = k; i < m; ++i) s += std::conj(v[i - k]) * Qh[(size_t)i * m + j];
      for (int i = k; i < m; ++i) Qh[(size_t)i * m + j] -= 2.0 * v[i - k] * s;
    }
  }
  // solve R[:n,:n] X = Qh[:n, :] (back substitution), X is n x m
  std::vector<cplx> X((size_t)n * m);
  for (int j = 0; j < m; ++j) {
    for (int i = n - 1; i >= 0; --i) {
      cplx s = Qh[(size_t)i * m + j];
      for (int l = i + 1; l < n; ++l) s -= R[(size_t)i * n + l] * X[(size_t)l * m + j];
      X[(size_t)i * m + j] = s / R[(size_t)i * n + i];
    }
  }
  return X;
}

sgw_status build_grid(sgw_ctx* c) {
  const int n = c->nt;
  const double beta = c->p.beta;
  c->tau.resize(n);
  std::vector<double> Cm((size_t)n * n);  // values -> Chebyshev coefficients
  for (int j = 0; j < n; ++j) {
    const double th = kPi * (j + 0.5) / n;
    c->tau[j] = 0.5 * beta * (1.0 - std::cos(th));
    for (int l = 0; l < n; ++l) {
      // x_j = -cos(th) = cos(pi - th), T_l(x_j) = cos(l (pi - th))
      Cm[(size_t)l * n + j] = (l == 0 ? 1.0 : 2.0) / n * std::cos(l * (kPi - th));
    }
  }
  auto forward = [&](const std::vector<int>& idx, bool fermi, std::vector<cplx>& T, std::vector<double>& nu) {
    const int m = (int)idx.size();
    T.assign((size_t)m * n, cplx(0, 0));
    nu.resize(m);
    std::vector<cplx> I;
    for (int r = 0; r < m; ++r) {
      const double v = fermi ? (2.0 * idx[r] + 1.0) * kPi / beta : 2.0 * idx[r] * kPi / beta;
      nu[r] = v;
      const double a = 0.5 * v * beta;
      const double zeta = fermi ? -1.0 : 1.0;
      fourier_cheb(a, n, zeta, I);
      // I_l(nu) = (beta/2) int_{-1}^{1} e^{i a (1+x)} T_l dx; the integration-by-parts branch
      // already includes the phase e^{ia}, the quadrature branch integrates e^{ia(1+x)} directly.
      for (int l = 0; l < n; ++l) {
        const cplx Il = 0.5 * beta * I[l];
        for (int j = 0; j < n; ++j) T[(size_t)r * n + j] += Il * Cm[(size_t)l * n + j];
      }
    }
  };
  forward(c->mats_f, true, c->TF, c->nu_f);
  forward(c->mats_b, false, c->TB, c->nu_b);
  c->TFbar = pinv_qr(c->TF, c->nwf, n);
  c->TBbar = pinv_qr(c->TB, c->nwb, n);
  c->beta_row.assign(n, 0.0);
  for (int j = 0; j < n; ++j)
    for (int l = 0; l < n; ++l) c->beta_row[j] += Cm[(size_t)l * n + j];
  c->gamma_w.assign(c->nwf, cplx(0, 0));
  for (int m = 0; m < c->nwf; ++m)
    for (int j = 0; j < n; ++j) c->gamma_w[m] -= c->beta_row[j] * c->TFbar[(size_t)j * c->nwf + m];
  std::vector<double> gx, gw;
  gauss_legendre(n, gx, gw);
  c->gl_interp.assign((size_t)n * n, 0.0);
  c->gl_w.resize(n);
  for (int g = 0; g < n; ++g) {
    c->gl_w[g] = gw[g];
    const double th = std::acos(gx[g]);
    for (int j = 0; j < n; ++j) {
      double s = 0;
      for (int l = 0; l < n; ++l) s += std::cos(l * th) * Cm[(size_t)l * n + j];
      c->gl_interp[(size_t)g * n + j] = s;
    }
  }
  return SGW_OK;
}

// ---------------------------------------------------------------------------
// Real spherical harmonics and their rotation matrices
// ---------------------------------------------------------------------------
static double real_ylm(int l, int m, double x, double y, double z) {
  const double r = std::sqrt(x * x + y * y + z * z);
  const double ct = z / r;
  const double st = std::sqrt(std::max(0.0, 1.0 - ct * ct));
  const double phi = std::atan2(y, x);
  const int am = std::abs(m);
  // associated Legendre P_l^am(ct) without the Condon-Shortley phase
  double pmm = 1.0;
  for (int i = 1; i <= am; ++i) pmm *= (2.0 * i - 1.0) * st;
  double plm = pmm;
  if (l > am) {
    double p1 = ct * (2.0 * am + 1.0) * pmm;
    double p0 = pmm;
    plm = p1;
    for (int ll = am + 2; ll <= l; ++ll) {
      const double p2 = ((2.0 * ll - 1.0) * ct * p1 - (ll + am - 1.0) * p0) / (ll - am);
      p0 = p1;
      p1 = p2;
      plm = p2;
    }
  }
  double fact = 1.0;  // (l-am)!/(l+am)!
  for (int i = l - am + 1; i <= l + am; ++i) fact /= i;
  const double N = std::sqrt((2.0 * l + 1.0) / (4.0 * kPi) * fact);
  if (m == 0) return N * plm;
  if (m > 0) return std::sqrt(2.0) * N * plm * std::cos(m * phi);
  return std::sqrt(2.0) * N * plm * std::sin(am * phi);
}

// D[m'][m] = int Y_lm'(u) Y_lm(R^T u) dOmega: exact product quadrature (Gauss-Legendre in
// cos(theta), trapezoid in phi) for the degree-2l integrand.
static std::vector<double> harmonic_rotation(int l, const double* R) {
  const int d = 2 * l + 1;
  std::vector<double> D((size_t)d * d, 0.0);
  std::vector<double> gx, gw;
  gauss_legendre(l + 2, gx, gw);
  const int nphi = 2 * l + 3;
  std::vector<double> ya(d), yb(d);
  for (size_t it = 0; it < gx.size(); ++it) {
    const double ct = gx[it], st = std::sqrt(1.0 - ct * ct);
    for (int ip = 0; ip < nphi; ++ip) {
      const double ph = 2.0 * kPi * (ip + 0.5) / nphi;
      const double u[3] = {st * std::cos(ph), st * std::sin(ph), ct};
      double v[3];  // R^T u
      for (int i = 0; i < 3; ++i) v[i] = R[0 * 3 + i] * u[0] + R[1 * 3 + i] * u[1] + R[2 * 3 + i] * u[2];
      const double wgt = gw[it] * 2.0 * kPi / nphi;
      for (int m = -l; m <= l; ++m) {
        ya[m + l] = real_ylm(l, m, u[0], u[1], u[2]);
        yb[m + l] = real_ylm(l, m, v[0], v[1], v[2]);
      }
      for (int a = 0; a < d; ++a)
        for (int b = 0; b < d; ++b) D[(size_t)a * d + b] += wgt * ya[a] * yb[b];
    }
  }
  return D;
}

// ---------------------------------------------------------------------------
// Hermitian Jacobi on the host (set-up only: the Dirac-character matrices are
// at most 2 (2l+1) wide).  Eigenvectors in the columns of V.
// ---------------------------------------------------------------------------
static void host_jacobi(std::vector<cplx>& A, int n, std::vector<cplx>& V, std::vector<double>& ev) {
  V.assign((size_t)n * n, cplx(0, 0));
  for (int i = 0; i < n; ++i) V[(size_t)i * n + i] = 1.0;
  for (int sweep = 0; sweep < 100; ++sweep) {
    double off = 0, tot = 0;
    for (int i = 0; i < n; ++i)
      for (int j = 0; j < n; ++j) {
        const double v = std::norm(A[(size_t)i * n + j]);
        tot += v;
        if (i != j) off += v;
      }
    if (!(off > 1e-30 * tot)) break;
    for (int p = 0; p < n; ++p)
      for (int q = p + 1; q < n; ++q) {
        const cplx apq = A[(size_t)p * n + q];
        const double b = std::abs(apq);
        if (b < 1e-300) continue;
        const cplx z = apq / b;
        const double tau = (A[(size_t)q * n + q].real() - A[(size_t)p * n + p].real()) / (2.0 * b);
        const double t = (tau >= 0 ? 1.0 : -1.0) / (std::fabs(tau) + std::sqrt(1.0 + tau * tau));
        const double cc = 1.0 / std::sqrt(1.0 + t * t), s = t * cc;
        for (int j = 0; j < n; ++j) {
          const cplx ap = A[(size_t)p * n + j], aq = A[(size_t)q * n + j];
          A[(size_t)p * n + j] = cc * ap - s * z * aq;
          A[(size_t)q * n + j] = s * ap + cc * z * aq;
        }
        for (int r = 0; r < n; ++r) {
          const cplx xp = A[(size_t)r * n + p], xq = std::conj(z) * A[(size_t)r * n + q];
          A[(size_t)r * n + p] = cc * xp - s * xq;
          A[(size_t)r * n + q] = s * xp + cc * xq;
          const cplx vp = V[(size_t)r * n + p], vq = std::conj(z) * V[(size_t)r * n + q];
          V[(size_t)r * n + p] = cc * vp - s * vq;
          V[(size_t)r * n + q] = s * vp + cc * vq;
        }
      }
  }
  ev.resize(n);
  for (int i = 0; i < n; ++i) ev[i] = A[(size_t)i * n + i].real();
}

// ---------------------------------------------------------------------------
// Space-group analysis
// ---------------------------------------------------------------------------
namespace {
struct Basis {
  std::vector<int> shells;
  int per_atom = 0, n = 0;
  std::vector<int> shell_off;
  std::map<int, std::vector<std::vector<double>>> D;  // l -> per op rotation matrix
};

void inv3(const double* A, double* B) {
  const double det = A[0] * (A[4] * A[8] - A[5] * A[7]) - A[1] * (A[3] * A[8] - A[5] * A[6]) +
                     A[2] * (A[3] * A[7] - A[4] * A[6]);
  B[0] = (A[4] * A[8] - A[5] * A[7]) / det;
  B[1] = (A[2] * A[7] - A[1] * A[8]) / det;
  B[2] = (A[1] * A[5] - A[2] * A[4]) / det;
  B[3] = (A[5] * A[6] - A[3] * A[8]) / det;
  B[4] = (A[0] * A[8] - A[2] * A[6]) / det;
  B[5] = (A[2] * A[3] - A[0] * A[5]) / det;
  B[6] = (A[3] * A[7] - A[4] * A[6]) / det;
  B[7] = (A[1] * A[6] - A[0] * A[7]) / det;
  B[8] = (A[0] * A[4] - A[1] * A[3]) / det;
}
void mul3(const double* A, const double* B, double* C) {
  for (int i = 0; i < 3; ++i)
    for (int j = 0; j < 3; ++j) C[i * 3 + j] = A[i * 3] * B[j] + A[i * 3 + 1] * B[3 + j] + A[i * 3 + 2] * B[6 + j];
}
}  // namespace

sgw_status build_symmetry(sgw_ctx* c, const sgw_structure* st) {
  const int nops = st->nops, nat = st->natom;
  const int n1 = c->p.nk[0], n2 = c->p.nk[1], n3 = c->p.nk[2];
  const int Nk = c->Nk;
  double A[9], Ai[9];
  std::memcpy(A, st->lattice, sizeof(A));
  inv3(A, Ai);
  // integer action on fractional k: M = A^T R A^{-T}
  std::vector<std::array<int, 9>> Mk(nops);
  for (int o = 0; o < nops; ++o) {
    const double* R = st->rotations + 9 * o;
    double At[9], AiT[9], T1[9], T2[9];
    for (int i = 0; i < 3; ++i)
      for (int j = 0; j < 3; ++j) { At[i * 3 + j] = A[j * 3 + i]; AiT[i * 3 + j] = Ai[j * 3 + i]; }
    mul3(At, R, T1);
    mul3(T1, AiT, T2);
    for (int i = 0; i < 9; ++i) {
      const double r = std::round(T2[i]);
      if (std::fabs(r - T2[i]) > 1e-8) return c->fail(SGW_ERR_ARG, "operation does not preserve the lattice");
      Mk[o][i] = (int)r;
    }
  }
  auto kidx = [&](int a, int b, int cc) {
    a = ((a % n1) + n1) % n1;
    b = ((b % n2) + n2) % n2;
    cc = ((cc % n3) + n3) % n3;
    return (a * n2 + b) * n3 + cc;
  };
  std::vector<std::array<int, 3>> iv(Nk);
  for (int a = 0; a < n1; ++a)
    for (int b = 0; b < n2; ++b)
      for (int cc = 0; cc < n3; ++cc) iv[kidx(a, b, cc)] = {a, b, cc};
  // image of k under op o; note n1 = n2 = n3 is required for a general cubic action
  std::vector<std::vector<int>> image(nops, std::vector<int>(Nk));
  std::vector<std::vector<std::array<double, 3>>> krot(nops, std::vector<std::array<double, 3>>(Nk));
  for (int o = 0; o < nops; ++o)
    for (int k = 0; k < Nk; ++k) {
      const double f[3] = {(double)iv[k][0] / n1, (double)iv[k][1] / n2, (double)iv[k][2] / n3};
      double g[3];
      for (int i = 0; i < 3; ++i) g[i] = Mk[o][i * 3] * f[0] + Mk[o][i * 3 + 1] * f[1] + Mk[o][i * 3 + 2] * f[2];
      krot[o][k] = {g[0], g[1], g[2]};
      const double ia = g[0] * n1, ib = g[1] * n2, ic = g[2] * n3;
      if (std::fabs(ia - std::round(ia)) > 1e-8 || std::fabs(ib - std::round(ib)) > 1e-8 ||
          std::fabs(ic - std::round(ic)) > 1e-8)
        return c->fail(SGW_ERR_ARG, "k mesh is not invariant under the operations");
      image[o][k] = kidx((int)std::lround(ia), (int)std::lround(ib), (int)std::lround(ic));
    }
  // identity must be op 0
  {
    const double* R = st->rotations;
    for (int i = 0; i < 9; ++i)
      if (std::fabs(R[i] - ((i % 4 == 0) ? 1.0 : 0.0)) > 1e-12)
        return c->fail(SGW_ERR_ARG, "operation 0 must be the identity");
  }
  // atom mapping: R r_x + v = r_x' + T
  std::vector<std::vector<int>> perm(nops, std::vector<int>(nat));
  std::vector<std::vector<std::array<double, 3>>> tvec(nops, std::vector<std::array<double, 3>>(nat));
  for (int o = 0; o < nops; ++o) {
    const double* R = st->rotations + 9 * o;
    const double* v = st->translations + 3 * o;
    for (int x = 0; x < nat; ++x) {
      const double* r = st->positions + 3 * x;
      double rp[3];
      for (int i = 0; i < 3; ++i) rp[i] = R[i * 3] * r[0] + R[i * 3 + 1] * r[1] + R[i * 3 + 2] * r[2] + v[i];
      int found = -1;
      for (int y = 0; y < nat && found < 0; ++y) {
        const double* ry = st->positions + 3 * y;
        double d[3] = {rp[0] - ry[0], rp[1] - ry[1], rp[2] - ry[2]}, t[3];
        for (int i = 0; i < 3; ++i) t[i] = Ai[i * 3] * d[0] + Ai[i * 3 + 1] * d[1] + Ai[i * 3 + 2] * d[2];
        bool ok = true;
        for (int i = 0; i < 3; ++i) ok = ok && std::fabs(t[i] - std::round(t[i])) < 1e-8;
        if (ok) {
          found = y;
          tvec[o][x] = {std::round(t[0]), std::round(t[1]), std::round(t[2])};
        }
      }
      if (found < 0) return c->fail(SGW_ERR_ARG, "operation does not map the crystal onto itself");
      perm[o][x] = found;
    }
  }
  // bases
  Basis bas[2];
  bas[0].shells.assign(st->ao_shells, st->ao_shells + st->n_ao_shells);
  bas[1].shells.assign(st->aux_shells, st->aux_shells + st->n_aux_shells);
  for (int b = 0; b < 2; ++b) {
    int o = 0;
    for (int l : bas[b].shells) {
      bas[b].shell_off.push_back(o);
      o += 2 * l + 1;
    }
    bas[b].per_atom = o;
    bas[b].n = o * nat;
    for (int l : bas[b].shells)
      if (!bas[b].D.count(l))
        for (int op = 0; op < nops; ++op) bas[b].D[l].push_back(harmonic_rotation(l, st->rotations + 9 * op));
  }
  if (bas[0].n != c->nao || bas[1].n != c->naux) return c->fail(SGW_ERR_ARG, "shell lists do not match nao / naux");

  // stars and wedge
  c->rep.assign(Nk, -1);
  c->op.assign(Nk, 0);
  c->wedge_k.clear();
  for (int k = 0; k < Nk; ++k) {
    if (c->rep[k] >= 0) continue;
    const int w = (int)c->wedge_k.size();
    c->wedge_k.push_back(k);
    for (int o = 0; o < nops; ++o) {
      const int kk = image[o][k];
      if (c->rep[kk] < 0) {
        c->rep[kk] = w;
        c->op[kk] = o;
      }
    }
  }
  c->nwedge = (int)c->wedge_k.size();
  c->star.assign(c->nwedge, 0);
  for (int k = 0; k < Nk; ++k) c->star[c->rep[k]]++;

  // phase of op o acting on a Bloch sum at k for atom x: exp(-2 pi i (M k) . t)
  auto phase = [&](int o, int k, int x) {
    const auto& g = krot[o][k];
    const auto& t = tvec[o][x];
    return std::exp(cplx(0.0, -2.0 * kPi * (g[0] * t[0] + g[1] * t[1] + g[2] * t[2])));
  };
  // Structured application of O^k(o) to the rows of a dense n x ncol matrix: Y = O X.
  auto apply_O = [&](const Basis& B, int o, int k, const std::vector<cplx>& X, int ncol, std::vector<cplx>& Y) {
    Y.assign((size_t)B.n * ncol, cplx(0, 0));
    for (int x = 0; x < nat; ++x) {
      const int xp = perm[o][x];
      const cplx ph = phase(o, k, x);
      for (size_t s = 0; s < B.shells.size(); ++s) {
        const int l = B.shells[s], d = 2 * l + 1;
        const auto& D = B.D.at(l)[o];
        const int src = x * B.per_atom + B.shell_off[s], dst = xp * B.per_atom + B.shell_off[s];
        for (int a = 0; a < d; ++a)
          for (int bb = 0; bb < d; ++bb) {
            const cplx f = ph * D[(size_t)a * d + bb];
            if (f == cplx(0, 0)) continue;
            for (int j = 0; j < ncol; ++j) Y[(size_t)(dst + a) * ncol + j] += f * X[(size_t)(src + bb) * ncol + j];
          }
      }
    }
  };

  // Partner-adapted basis of every block of the Dirac basis U (Sec. 3.4): a block of irrep dimension d
  // and multiplicity m holds m copies of the irrep.  Gamma(g) = U_b^dagger D(g) U_b is the
  // representation on the block.  A group-averaged random Hermitian operator
  // A1 = (1/h) sum_g Gamma R1 Gamma^dagger commutes with it, so it is I_d (x) a on the copies:
  // its eigenvalues come in m clusters of d, one cluster per copy.  A second averaged operator A2
  // maps copy 1 onto copy a through T_a = C_a^dagger A2 C_1.  By Schur's lemma T_a is a scalar times
  // a unitary W_a, and the basis C_a W_a of copy a transforms exactly as C_1 does.  The columns are
  // ordered partner-major, (partner i, copy a) at i m + a, so every invariant operator reads I_d (x) A
  // on the block.  A block with d = 1, an invalid d, or clusters not of size d keeps its Dirac basis.
  auto partner_basis = [&](const Basis& B, const std::vector<cplx>& U, const Partition& P, const std::vector<int>& bstart,
                           int w, int fam, int k, const std::vector<int>& little, auto&& kv, auto&& applyO) {
    const int n = B.n, h = (int)little.size();
    std::vector<cplx> Up(U);
    std::vector<std::vector<cplx>> DU(h);
    for (int i = 0; i < h; ++i) {
      applyO(B, little[i], k, U, n, DU[i]);
      const cplx e = kv(little[i]);
      for (auto& z : DU[i]) z *= e;
    }
    std::mt19937_64 rng(0x5eed0000ULL + 131ULL * w + 7ULL * fam);
    auto unif = [&]() { return (double)(rng() >> 11) * (1.0 / 9007199254740992.0) - 0.5; };
    for (size_t bi = 0; bi < P.sizes.size(); ++bi) {
      const int sz = P.sizes[bi], d = P.dims[bi], b0 = bstart[bi];
      if (d <= 1 || sz % d != 0) continue;
      const int m = sz / d;
      std::vector<std::vector<cplx>> Gm(h, std::vector<cplx>((size_t)sz * sz));
      for (int i = 0; i < h; ++i)
        for (int r = 0; r < sz; ++r)
          for (int cc = 0; cc < sz; ++cc) {
            cplx acc(0, 0);
            for (int t = 0; t < n; ++t) acc += std::conj(U[(size_t)t * n + b0 + r]) * DU[i][(size_t)t * n + b0 + cc];
            Gm[i][(size_t)r * sz + cc] = acc;
          }
      auto average = [&](const std::vector<cplx>& R) {
        std::vector<cplx> A((size_t)sz * sz, cplx(0, 0)), T((size_t)sz * sz);
        for (int i = 0; i < h; ++i) {
          const auto& Gg = Gm[i];
          for (int r = 0; r < sz; ++r)
            for (int cc = 0; cc < sz; ++cc) {
              cplx acc(0, 0);
              for (int t = 0; t < sz; ++t) acc += Gg[(size_t)r * sz + t] * R[(size_t)t * sz + cc];
              T[(size_t)r * sz + cc] = acc;
            }
          for (int r = 0; r < sz; ++r)
            for (int cc = 0; cc < sz; ++cc) {
              cplx acc(0, 0);
              for (int t = 0; t < sz; ++t) acc += T[(size_t)r * sz + t] * std::conj(Gg[(size_t)cc * sz + t]);
              A[(size_t)r * sz + cc] += acc;
            }
        }
        for (auto& z : A) z /= (double)h;
        return A;
      };
      std::vector<cplx> R1((size_t)sz * sz), R2((size_t)sz * sz);
      for (int r = 0; r < sz; ++r)
        for (int cc = 0; cc <= r; ++cc) {
          const cplx z(unif(), r == cc ? 0.0 : unif());
          R1[(size_t)r * sz + cc] = z;
          R1[(size_t)cc * sz + r] = std::conj(z);
        }
      for (auto& z : R2) z = cplx(unif(), unif());
      std::vector<cplx> A1 = average(R1), A2 = average(R2);
      std::vector<cplx> V;
      std::vector<double> ev;
      host_jacobi(A1, sz, V, ev);
      std::vector<int> ord(sz);
      std::iota(ord.begin(), ord.end(), 0);
      std::sort(ord.begin(), ord.end(), [&](int a, int bb) { return ev[a] < ev[bb]; });
      double scale = 0.0;
      for (double e : ev) scale = std::max(scale, std::fabs(e));
      bool ok = true;
      for (int a = 0; a < m && ok; ++a) {  // clusters of exactly d, separated from their neighbours
        const double lo = ev[ord[a * d]], hi = ev[ord[a * d + d - 1]];
        ok = hi - lo <= 1e-9 * scale && (a == 0 || lo - ev[ord[a * d - 1]] > 1e-7 * scale);
      }
      if (!ok) continue;
      // C[a] column j = V[:, ord[a d + j]]; T_a = C_a^dagger A2 C_1; W_a = T_a / sqrt(tr(T^dagger T) / d)
      std::vector<cplx> blk((size_t)sz * sz, cplx(0, 0));  // new basis in block coordinates, column i m + a
      for (int a = 0; a < m; ++a) {
        std::vector<cplx> W((size_t)d * d, cplx(0, 0));
        if (a == 0) {
          for (int i = 0; i < d; ++i) W[(size_t)i * d + i] = 1.0;
        } else {
          std::vector<cplx> A2C1((size_t)sz * d, cplx(0, 0));
          for (int r = 0; r < sz; ++r)
            for (int j = 0; j < d; ++j) {
              cplx acc(0, 0);
              for (int t = 0; t < sz; ++t) acc += A2[(size_t)r * sz + t] * V[(size_t)t * sz + ord[j]];
              A2C1[(size_t)r * d + j] = acc;
            }
          double nrm = 0.0;
          for (int i = 0; i < d; ++i)
            for (int j = 0; j < d; ++j) {
              cplx acc(0, 0);
              for (int r = 0; r < sz; ++r) acc += std::conj(V[(size_t)r * sz + ord[a * d + i]]) * A2C1[(size_t)r * d + j];
              W[(size_t)i * d + j] = acc;
              nrm += std::norm(acc);
            }
          nrm = std::sqrt(nrm / d);
          if (!(nrm > 1e-12 * std::max(1.0, scale))) { ok = false; break; }
          for (auto& z : W) z /= nrm;
        }
        // copy a's new partner i = sum_j C_a[:, j] W[j][i]
        for (int i = 0; i < d; ++i)
          for (int r = 0; r < sz; ++r) {
            cplx acc(0, 0);
            for (int j = 0; j < d; ++j) acc += V[(size_t)r * sz + ord[a * d + j]] * W[(size_t)j * d + i];
            blk[(size_t)r * sz + (size_t)i * m + a] = acc;
          }
      }
      if (!ok) continue;
      for (int t = 0; t < n; ++t)
        for (int col = 0; col < sz; ++col) {
          cplx acc(0, 0);
          for (int r = 0; r < sz; ++r) acc += U[(size_t)t * n + b0 + r] * blk[(size_t)r * sz + col];
          Up[(size_t)t * n + b0 + col] = acc;
        }
    }
    return Up;
  };

  // irrep bases at the wedge points
  std::vector<std::vector<cplx>> Uw[2];
  c->part_ao.assign(c->nwedge, Partition());
  c->part_aux.assign(c->nwedge, Partition());
  for (int b = 0; b < 2; ++b) Uw[b].assign(c->nwedge, {});
  for (int w = 0; w < c->nwedge; ++w) {
    const int k = c->wedge_k[w];
    std::vector<int> little;
    for (int o = 0; o < nops; ++o)
      if (image[o][k] == k) little.push_back(o);
    const int h = (int)little.size();
    // group product on rotation parts: index of R_a R_b inside the little group
    auto find_rot = [&](const double* R) {
      for (int i = 0; i < h; ++i) {
        const double* Q = st->rotations + 9 * little[i];
        bool eq = true;
        for (int j = 0; j < 9 && eq; ++j) eq = std::fabs(Q[j] - R[j]) < 1e-9;
        if (eq) return i;
      }
      return -1;
    };
    std::vector<int> inv(h), prod((size_t)h * h);
    for (int i = 0; i < h; ++i)
      for (int j = 0; j < h; ++j) {
        double P[9];
        mul3(st->rotations + 9 * little[i], st->rotations + 9 * little[j], P);
        const int r = find_rot(P);
        if (r < 0) return c->fail(SGW_ERR_ARG, "little co-group is not closed");
        prod[(size_t)i * h + j] = r;
        if (r == 0) inv[i] = j;
      }
    // conjugacy classes
    std::vector<int> cls(h, -1);
    std::vector<int> reps;
    for (int g = 0; g < h; ++g) {
      if (cls[g] >= 0) continue;
      const int id = (int)reps.size();
      reps.push_back(g);
      for (int bt = 0; bt < h; ++bt) cls[prod[(size_t)prod[(size_t)bt * h + g] * h + inv[bt]]] = id;
    }
    const int ncls = (int)reps.size();
    std::vector<int> ncl(ncls, 0);
    for (int g = 0; g < h; ++g) ncl[cls[g]]++;
    // e^{i k . v} with k . v = 2 pi kfrac . (A^{-1} v)
    const double kf[3] = {(double)iv[k][0] / n1, (double)iv[k][1] / n2, (double)iv[k][2] / n3};
    auto kv = [&](int o) {
      const double* v = st->translations + 3 * o;
      double t[3];
      for (int i = 0; i < 3; ++i) t[i] = Ai[i * 3] * v[0] + Ai[i * 3 + 1] * v[1] + Ai[i * 3 + 2] * v[2];
      return std::exp(cplx(0.0, 2.0 * kPi * (kf[0] * t[0] + kf[1] * t[1] + kf[2] * t[2])));
    };
    for (int b = 0; b < 2; ++b) {
      const Basis& B = bas[b];
      struct Vec {
        double ev;
        int shell, dim;
        std::vector<cplx> v;  // over (x, m) of that shell
      };
      struct Eig {
        std::vector<double> ev;
        std::vector<cplx> V;
        std::vector<int> dim;
      };
      std::vector<Vec> all;
      std::map<int, Eig> by_l;
      for (auto& kvp : B.D) {
        const int l = kvp.first, d = 2 * l + 1, ds = nat * d;
        // projective representation D^k(a) = e^{i k.v(a)} O^k(a) on the subspace of one shell of angular momentum l
        std::vector<std::vector<cplx>> Dm(h, std::vector<cplx>((size_t)ds * ds, cplx(0, 0)));
        for (int i = 0; i < h; ++i) {
          const int o = little[i];
          const cplx e = kv(o);
          const auto& D = kvp.second[o];
          for (int x = 0; x < nat; ++x) {
            const int xp = perm[o][x];
            const cplx ph = e * phase(o, k, x);
            for (int a = 0; a < d; ++a)
              for (int bb = 0; bb < d; ++bb) Dm[i][(size_t)(xp * d + a) * ds + x * d + bb] = ph * D[(size_t)a * d + bb];
          }
        }
        // Dirac characters Omega_c = (n_c / h) sum_beta D(beta) D(gamma_c) D(beta)^dagger, and the
        // Hermitian combination H = sum_c a_c (Omega + Omega^dagger) + b_c i (Omega - Omega^dagger)
        std::vector<cplx> Hm((size_t)ds * ds, cplx(0, 0)), T1((size_t)ds * ds), Om((size_t)ds * ds);
        std::vector<std::vector<cplx>> Oms(ncls);
        for (int cc = 0; cc < ncls; ++cc) {
          std::fill(Om.begin(), Om.end(), cplx(0, 0));
          const auto& Dg = Dm[reps[cc]];
          for (int bt = 0; bt < h; ++bt) {
            const auto& Db = Dm[bt];
            for (int i = 0; i < ds; ++i)
              for (int j = 0; j < ds; ++j) {
                cplx s(0, 0);
                for (int l2 = 0; l2 < ds; ++l2) s += Db[(size_t)i * ds + l2] * Dg[(size_t)l2 * ds + j];
                T1[(size_t)i * ds + j] = s;
              }
            for (int i = 0; i < ds; ++i)
              for (int j = 0; j < ds; ++j) {
                cplx s(0, 0);
                for (int l2 = 0; l2 < ds; ++l2) s += T1[(size_t)i * ds + l2] * std::conj(Db[(size_t)j * ds + l2]);
                Om[(size_t)i * ds + j] += s * ((double)ncl[cc] / h);
              }
          }
          Oms[cc] = Om;
          const double ac = std::sin(1.0 + 2.3 * cc) + 1.7, bc = std::cos(0.5 + 1.3 * cc);
          for (int i = 0; i < ds; ++i)
            for (int j = 0; j < ds; ++j) {
              const cplx o1 = Om[(size_t)i * ds + j], o2 = std::conj(Om[(size_t)j * ds + i]);
              Hm[(size_t)i * ds + j] += ac * (o1 + o2) + bc * cplx(0, 1) * (o1 - o2);
            }
        }
        std::vector<cplx> V;
        std::vector<double> ev;
        host_jacobi(Hm, ds, V, ev);
        // irrep dimension of each eigenvector: on an irrep subspace Omega_c acts as
        // lambda_c = n_c chi(gamma_c) / d, |chi| is constant on a class (conjugation adds a phase
        // in a projective representation), and sum_g |chi(g)|^2 = h, so
        // d^2 = h / sum_c |lambda_c|^2 / n_c with lambda_c the Rayleigh quotient v^dagger Omega_c v
        std::vector<int> dim(ds, 0);
        for (int j = 0; j < ds; ++j) {
          double sum = 0.0;
          for (int cc = 0; cc < ncls; ++cc) {
            cplx lam(0, 0);
            for (int i = 0; i < ds; ++i) {
              cplx t(0, 0);
              for (int k2 = 0; k2 < ds; ++k2) t += Oms[cc][(size_t)i * ds + k2] * V[(size_t)k2 * ds + j];
              lam += std::conj(V[(size_t)i * ds + j]) * t;
            }
            sum += std::norm(lam) / ncl[cc];
          }
          dim[j] = sum > 0.0 ? (int)std::lround(std::sqrt((double)h / sum)) : 0;
        }
        by_l[l] = {ev, V, dim};
      }
      for (size_t s = 0; s < B.shells.size(); ++s) {
        const int l = B.shells[s], d = 2 * l + 1, ds = nat * d;
        const Eig& evV = by_l[l];
        for (int j = 0; j < ds; ++j) {
          Vec vv;
          vv.ev = evV.ev[j];
          vv.shell = (int)s;
          vv.dim = evV.dim[j];
          vv.v.resize(ds);
          for (int i = 0; i < ds; ++i) vv.v[i] = evV.V[(size_t)i * ds + j];
          all.push_back(vv);
        }
      }
      std::stable_sort(all.begin(), all.end(), [](const Vec& a, const Vec& b) { return a.ev < b.ev; });
      double scale = 1.0;
      for (auto& v : all) scale = std::max(scale, std::fabs(v.ev));
      const double tol = 1e-7 * scale;
      Partition P;
      std::vector<cplx> U((size_t)B.n * B.n, cplx(0, 0));
      int col = 0, start = 0;
      for (size_t i = 0; i < all.size(); ++i) {
        if (i > 0 && all[i].ev - all[i - 1].ev > tol) {
          if (all[i].ev - all[i - 1].ev < 1e-4 * scale)
            return c->fail(SGW_ERR_ARG, "Dirac-character eigenvalues of distinct irreps are too close");
          P.sizes.push_back(col - start);
          start = col;
        }
        if (col == start) P.dims.push_back(all[i].dim);
        else if (P.dims.back() != all[i].dim) P.dims.back() = 0;
        const int s = all[i].shell, l = B.shells[s], d = 2 * l + 1;
        for (int x = 0; x < nat; ++x)
          for (int a = 0; a < d; ++a)
            U[(size_t)(x * B.per_atom + B.shell_off[s] + a) * B.n + col] = all[i].v[x * d + a];
        ++col;
      }
      P.sizes.push_back(col - start);
      long long off = 0;
      int st0 = 0;
      std::vector<int> bstart;
      std::vector<long long> bdoff;
      for (int sz : P.sizes) {
        bstart.push_back(st0);
        bdoff.push_back(off);
        st0 += sz;
        off += (long long)sz * sz;
      }
      P.elems = off;
      P.starts.resize(B.n);
      P.doff.resize(B.n);
      std::vector<int> vsize(B.n);
      for (size_t bi = 0; bi < P.sizes.size(); ++bi)
        for (int v = bstart[bi]; v < bstart[bi] + P.sizes[bi]; ++v) {
          P.starts[v] = bstart[bi];
          P.doff[v] = bdoff[bi];
          vsize[v] = P.sizes[bi];
        }
      P.isize = vsize;
      (b == 0 ? c->part_ao : c->part_aux)[w] = P;
      Uw[b][w] = U;
      if (c->want_partner) {
        if (c->partner_U[b].size() != (size_t)c->nwedge) c->partner_U[b].assign(c->nwedge, {});
        c->partner_U[b][w] = partner_basis(B, U, P, bstart, w, b, k, little, kv, apply_O);
      }
    }
  }
  // packed offsets
  c->g_off.assign(c->nwedge, 0);
  c->p_off.assign(c->nwedge, 0);
  long long go = 0, po = 0;
  c->max_ao_block = c->max_aux_block = 0;
  for (int w = 0; w < c->nwedge; ++w) {
    c->g_off[w] = go;
    c->p_off[w] = po;
    go += c->part_ao[w].elems;
    po += c->part_aux[w].elems;
    for (int s : c->part_ao[w].sizes) c->max_ao_block = std::max(c->max_ao_block, s);
    for (int s : c->part_aux[w].sizes) c->max_aux_block = std::max(c->max_aux_block, s);
  }
  c->g_elems = go;
  c->p_elems = po;

  // rotated bases U^k = O^{k_w}(a_k) U^{k_w} for every k
  std::vector<cplx> hostU[2];
  for (int b = 0; b < 2; ++b) {
    const int n = bas[b].n;
    hostU[b].assign((size_t)Nk * n * n, cplx(0, 0));
    std::vector<cplx> Y;
    for (int k = 0; k < Nk; ++k) {
      const int w = c->rep[k];
      apply_O(bas[b], c->op[k], c->wedge_k[w], Uw[b][w], n, Y);
      std::copy(Y.begin(), Y.end(), hostU[b].begin() + (size_t)k * n * n);
    }
  }
  // pairs
  for (int o = 0; o < 2; ++o) {
    c->pair_k1[o].clear();
    c->pair_k2[o].clear();
  }
  for (int w = 0; w < c->nwedge; ++w)
    for (int k = 0; k < Nk; ++k) {
      const int q = c->wedge_k[w];
      c->pair_k1[0].push_back(k);
      c->pair_k2[0].push_back(kidx(iv[k][0] + iv[q][0], iv[k][1] + iv[q][1], iv[k][2] + iv[q][2]));
      c->pair_k1[1].push_back(c->wedge_k[w]);
      c->pair_k2[1].push_back(k);
    }
  c->hostU[0].swap(hostU[0]);
  c->hostU[1].swap(hostU[1]);
  return SGW_OK;
}

}  // namespace sgw
