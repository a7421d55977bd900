// Device kernels of the plain (complex128) form.
//
// On GB300 the FP64 pipe issues about two fused multiply-adds per clock per SM
// (1.2 TFLOP/s for the chip), so every kernel here is bound by FP64 issue, not
// by memory: the designs keep all lanes busy with useful multiply-adds
// (thread-per-output loops over the actual block, split-K for small blocks)
// and read operands through L1/shared memory with coalesced rows.
#include <cfloat>
#include <cstdio>
#include <type_traits>

#include "sgw_internal.h"

namespace sgw {

__device__ __forceinline__ double2 cadd(double2 a, double2 b) { return make_double2(a.x + b.x, a.y + b.y); }
__device__ __forceinline__ double2 cmul(double2 a, double2 b) {
  return make_double2(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x);
}
// c + a * b
__device__ __forceinline__ double2 cfma(double2 a, double2 b, double2 c) {
  c.x = fma(a.x, b.x, c.x);
  c.x = fma(-a.y, b.y, c.x);
  c.y = fma(a.x, b.y, c.y);
  c.y = fma(a.y, b.x, c.y);
  return c;
}
// c + a * conj(b)
__device__ __forceinline__ double2 cfma_cj(double2 a, double2 b, double2 c) {
  c.x = fma(a.x, b.x, c.x);
  c.x = fma(a.y, b.y, c.x);
  c.y = fma(a.y, b.x, c.y);
  c.y = fma(-a.x, b.y, c.y);
  return c;
}
__device__ __forceinline__ double2 cconj(double2 a) { return make_double2(a.x, -a.y); }
__device__ __forceinline__ double cabs2(double2 a) { return a.x * a.x + a.y * a.y; }

// single-precision counterparts (chosen form: FP32 operands, FP32 accumulation)
__device__ __forceinline__ float2 cadd(float2 a, float2 b) { return make_float2(a.x + b.x, a.y + b.y); }
__device__ __forceinline__ float2 cmul(float2 a, float2 b) {
  return make_float2(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x);
}
__device__ __forceinline__ float2 cfma(float2 a, float2 b, float2 c) {
  c.x = fmaf(a.x, b.x, c.x);
  c.x = fmaf(-a.y, b.y, c.x);
  c.y = fmaf(a.x, b.y, c.y);
  c.y = fmaf(a.y, b.x, c.y);
  return c;
}
__device__ __forceinline__ float2 cfma_cj(float2 a, float2 b, float2 c) {
  c.x = fmaf(a.x, b.x, c.x);
  c.x = fmaf(a.y, b.y, c.x);
  c.y = fmaf(a.y, b.x, c.y);
  c.y = fmaf(-a.x, b.y, c.y);
  return c;
}
template <typename Z> __device__ __forceinline__ Z czero();
template <> __device__ __forceinline__ double2 czero<double2>() { return make_double2(0.0, 0.0); }
template <> __device__ __forceinline__ float2 czero<float2>() { return make_float2(0.f, 0.f); }
__device__ __forceinline__ double2 to_z(double2 a, double2) { return a; }
__device__ __forceinline__ float2 to_z(double2 a, float2) { return make_float2((float)a.x, (float)a.y); }

static inline unsigned grid_for(long long work, int threads, long long cap = 1 << 20) {
  long long b = (work + threads - 1) / threads;
  if (b < 1) b = 1;
  if (b > cap) b = cap;
  return (unsigned)b;
}

// ---------------------------------------------------------------------------
// Block-diagonal multiply.  For every item:
//   left : Y[u][v][w] = s * sum_{v' in blk(v)} M[v][v'] X[u][v'][w]
//   right: Y[u][v][w] = s * sum_{w' in blk(w)} X[u][v][w'] M[w'][w]
// M is the packed block-diagonal matrix of one wedge point (blocks row-major);
// trans/conj select M^T / conj(M).  One thread per output element, looping
// over exactly the elements of its block: no padding work for uneven blocks.
// ---------------------------------------------------------------------------
// Sign flips as integer operations (no FP pipe slot).
__device__ __forceinline__ double negd(double x) {
  return __longlong_as_double(__double_as_longlong(x) ^ (long long)0x8000000000000000ULL);
}
__device__ __forceinline__ float negd(float x) { return __int_as_float(__float_as_int(x) ^ (int)0x80000000u); }
template <typename Z>
__device__ __forceinline__ Z make_neg(Z a) {
  a.x = negd(a.x);
  a.y = negd(a.y);
  return a;
}
// scale class by bit pattern: 0 = +1, 1 = -1, 2 = general
__device__ __forceinline__ int scale_kind(double2 s) {
  const long long xb = __double_as_longlong(s.x), yb = __double_as_longlong(s.y);
  if ((yb & 0x7FFFFFFFFFFFFFFFLL) != 0) return 2;
  if (xb == 0x3FF0000000000000LL) return 0;
  if (xb == (long long)0xBFF0000000000000ULL) return 1;
  return 2;
}

// LEFT/TRANS/CONJ are compile-time so the inner loop holds nothing but loads and the four
// FMAs of a complex multiply-add (the FP64 pipe is the bound: no compare, negate or scale in it).
template <typename Z, int LEFT, int TRANS, int CONJ>
__global__ void __launch_bounds__(256) k_bd_mult(BdGeom g, const Z* __restrict__ X, Z* __restrict__ Y,
                                                 const Z* __restrict__ M, const BdItem* __restrict__ items,
                                                 long long nitems, const int* __restrict__ ps,
                                                 const int* __restrict__ pz, const long long* __restrict__ pd) {
  const int VW = g.Vd * g.Wd;
  const int E = g.U * VW;
  for (long long it = blockIdx.y; it < nitems; it += gridDim.y) {
    const BdItem item = items[it];
    const int sk = scale_kind(item.scale);
    const int* bs = ps + (long long)item.part * g.n_part;
    const int* bz = pz + (long long)item.part * g.n_part;
    const long long* bd = pd + (long long)item.part * g.n_part;
    for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < E; e += gridDim.x * blockDim.x) {
      // block-major output order: the outputs that use one diagonal block of M are consecutive,
      // so the lanes of a warp share one block size and run loops of equal length
      int u, v, w;
      if (LEFT) {
        // block of rows [st, st + n): outputs (u, v, w) with w fastest, then v, then u
        const int UW = g.U * g.Wd;
        const int cs = e / UW;  // a row of the block holding output e
        const int st = bs[cs], n = bz[cs];
        const int r2 = e - st * UW;
        u = r2 / (n * g.Wd);
        const int rem = r2 - u * n * g.Wd;
        const int lv = rem / g.Wd;
        v = st + lv;
        w = rem - lv * g.Wd;
      } else {
        // block of columns [st, st + n): outputs (u, v, w) with w fastest, then v (per u)
        u = e / VW;
        const int r = e - u * VW;
        const int cs = r / g.Vd;  // a column of the block holding output r
        const int st = bs[cs], n = bz[cs];
        const int r2 = r - st * g.Vd;
        v = r2 / n;
        w = st + (r2 - v * n);
      }
      Z acc = czero<Z>();
      if (LEFT) {
        const int st = bs[v], n = bz[v];
        const Z* Mb = M + item.m_off + bd[v];
        const int lv = v - st;
        const Z* Xp = X + item.x_off + (long long)u * g.xs_u + w + (long long)st * g.xs_v;
        const Z* mp = TRANS ? Mb + lv : Mb + (long long)lv * n;
        const long long ms = TRANS ? n : 1;
        for (int j = 0; j < n; ++j) {
          const Z m = mp[j * ms];
          acc = CONJ ? cfma_cj(Xp[(long long)j * g.xs_v], m, acc) : cfma(m, Xp[(long long)j * g.xs_v], acc);
        }
      } else {
        const int st = bs[w], n = bz[w];
        const Z* Mb = M + item.m_off + bd[w];
        const int lw = w - st;
        const Z* Xp = X + item.x_off + (long long)u * g.xs_u + (long long)v * g.xs_v + st;
        const Z* mp = TRANS ? Mb + (long long)lw * n : Mb + lw;
        const long long ms = TRANS ? 1 : n;
        for (int j = 0; j < n; ++j) {
          const Z m = mp[j * ms];
          acc = CONJ ? cfma_cj(Xp[j], m, acc) : cfma(Xp[j], m, acc);
        }
      }
      if (sk == 1) {
        acc.x = negd(acc.x);
        acc.y = negd(acc.y);
      } else if (sk == 2) {
        acc = cmul(to_z(item.scale, acc), acc);
      }
      Z* yp = Y + item.y_off + (long long)u * g.ys_u + (long long)v * g.ys_v + w;
      if (g.accumulate) acc = cadd(*yp, acc);
      *yp = acc;
    }
  }
}

template <typename Z>
static void bd_mult_t(const BdGeom& g, const Z* X, Z* Y, const Z* M, const BdItem* items, long long nitems,
                      const int* p_start, const int* p_size, const long long* p_doff, cudaStream_t st) {
  if (nitems <= 0) return;
  const long long E = (long long)g.U * g.Vd * g.Wd;
  unsigned bx = grid_for(E, 256, 4096);
  long long by = 65535;
  long long want = (8192 + bx - 1) / bx;
  if (want < by) by = want;
  if (by > nitems) by = nitems;
  if (by < 1) by = 1;
  const dim3 grid(bx, (unsigned)by);
  const int key = (g.left ? 4 : 0) | (g.trans ? 2 : 0) | (g.conj ? 1 : 0);
  switch (key) {
    case 0: k_bd_mult<Z, 0, 0, 0><<<grid, 256, 0, st>>>(g, X, Y, M, items, nitems, p_start, p_size, p_doff); break;
    case 1: k_bd_mult<Z, 0, 0, 1><<<grid, 256, 0, st>>>(g, X, Y, M, items, nitems, p_start, p_size, p_doff); break;
    case 2: k_bd_mult<Z, 0, 1, 0><<<grid, 256, 0, st>>>(g, X, Y, M, items, nitems, p_start, p_size, p_doff); break;
    case 3: k_bd_mult<Z, 0, 1, 1><<<grid, 256, 0, st>>>(g, X, Y, M, items, nitems, p_start, p_size, p_doff); break;
    case 4: k_bd_mult<Z, 1, 0, 0><<<grid, 256, 0, st>>>(g, X, Y, M, items, nitems, p_start, p_size, p_doff); break;
    case 5: k_bd_mult<Z, 1, 0, 1><<<grid, 256, 0, st>>>(g, X, Y, M, items, nitems, p_start, p_size, p_doff); break;
    case 6: k_bd_mult<Z, 1, 1, 0><<<grid, 256, 0, st>>>(g, X, Y, M, items, nitems, p_start, p_size, p_doff); break;
    default: k_bd_mult<Z, 1, 1, 1><<<grid, 256, 0, st>>>(g, X, Y, M, items, nitems, p_start, p_size, p_doff); break;
  }
}
void bd_mult(const BdGeom& g, const double2* X, double2* Y, const double2* M, const BdItem* items, long long nitems,
             const int* p_start, const int* p_size, const long long* p_doff, cudaStream_t st) {
  bd_mult_t<double2>(g, X, Y, M, items, nitems, p_start, p_size, p_doff, st);
}
void bd_mult(const BdGeom& g, const float2* X, float2* Y, const float2* M, const BdItem* items, long long nitems,
             const int* p_start, const int* p_size, const long long* p_doff, cudaStream_t st) {
  bd_mult_t<float2>(g, X, Y, M, items, nitems, p_start, p_size, p_doff, st);
}

// ---------------------------------------------------------------------------
// Block-diagonal multiply, chunked.  A work unit is (row, block b, chunk of <= 8 outputs
// inside b); the thread loads each element of its operand segment once and applies it to
// all outputs of its chunk (8 multiply-adds per load), and the index arithmetic is paid
// once per unit instead of once per output.
//   right: Y[u][v][w0+l] = s * sum_j X[u][v][st+j] M[j][w0-st+l]          (unit over w)
//   left : Y[u][v0+l][w] = s * sum_j M[v0-st+l][j] X[u][st+j][w]          (unit over v)
// Units of partition p: ustart/ucnt/ubst/ubn/udoff[p * ustride + i], i < nunits[p].
// ---------------------------------------------------------------------------
constexpr int kChunk = 8;

template <typename Z>
__global__ void __launch_bounds__(256) k_bd_mult2(BdGeom g, const Z* __restrict__ X, Z* __restrict__ Y,
                                                  const Z* __restrict__ M, const BdItem* __restrict__ items,
                                                  long long nitems, const int* __restrict__ nunits,
                                                  const int4* __restrict__ units, const long long* __restrict__ udoff,
                                                  int ustride) {
  for (long long it = blockIdx.y; it < nitems; it += gridDim.y) {
    const BdItem item = items[it];
    const int sk = scale_kind(item.scale);
    const int nu = nunits[item.part];
    const int4* up = units + (long long)item.part * ustride;
    const long long* dp = udoff + (long long)item.part * ustride;
    const Z* Xb = X + item.x_off;
    Z* Yb = Y + item.y_off;
    const Z* Mb = M + item.m_off;
    if (!g.left) {
      // rows (u, v), units over w
      const int rows = g.U * g.Vd;
      const long long E = (long long)rows * nu;
      for (long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x; e < E; e += (long long)gridDim.x * blockDim.x) {
        const int row = (int)(e / nu), ui = (int)(e - (long long)row * nu);
        const int u = row / g.Vd, v = row - u * g.Vd;
        const int4 un = up[ui];  // x: first output, y: count, z: block start, w: block size
        const Z* Mblk = Mb + dp[ui];
        const Z* xr = Xb + (long long)u * g.xs_u + (long long)v * g.xs_v + un.z;
        const int lw0 = un.x - un.z;
        Z acc[kChunk];
#pragma unroll
        for (int l = 0; l < kChunk; ++l) acc[l] = czero<Z>();
        for (int j = 0; j < un.w; ++j) {
          const Z x = xr[j];
#pragma unroll
          for (int l = 0; l < kChunk; ++l) {
            if (l < un.y) {
              Z m = g.trans ? Mblk[(long long)(lw0 + l) * un.w + j] : Mblk[(long long)j * un.w + lw0 + l];
              if (g.conj) m.y = -m.y;
              acc[l] = cfma(x, m, acc[l]);
            }
          }
        }
        Z* yr = Yb + (long long)u * g.ys_u + (long long)v * g.ys_v + un.x;
        const Z sc = to_z(item.scale, acc[0]);
#pragma unroll
        for (int l = 0; l < kChunk; ++l)
          if (l < un.y) {
            Z r = sk == 0 ? acc[l] : sk == 1 ? make_neg(acc[l]) : cmul(sc, acc[l]);
            if (g.accumulate) r = cadd(yr[l], r);
            yr[l] = r;
          }
      }
    } else {
      // units over v, then w fastest (coalesced along w)
      const long long E = (long long)g.U * nu * g.Wd;
      for (long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x; e < E; e += (long long)gridDim.x * blockDim.x) {
        const int w = (int)(e % g.Wd);
        const long long r = e / g.Wd;
        const int ui = (int)(r % nu), u = (int)(r / nu);
        const int4 un = up[ui];
        const Z* Mblk = Mb + dp[ui];
        const Z* xc = Xb + (long long)u * g.xs_u + (long long)un.z * g.xs_v + w;
        const int lv0 = un.x - un.z;
        Z acc[kChunk];
#pragma unroll
        for (int l = 0; l < kChunk; ++l) acc[l] = czero<Z>();
        for (int j = 0; j < un.w; ++j) {
          const Z x = xc[(long long)j * g.xs_v];
#pragma unroll
          for (int l = 0; l < kChunk; ++l) {
            if (l < un.y) {
              Z m = g.trans ? Mblk[(long long)j * un.w + lv0 + l] : Mblk[(long long)(lv0 + l) * un.w + j];
              if (g.conj) m.y = -m.y;
              acc[l] = cfma(m, x, acc[l]);
            }
          }
        }
        Z* yc = Yb + (long long)u * g.ys_u + (long long)un.x * g.ys_v + w;
        const Z sc = to_z(item.scale, acc[0]);
#pragma unroll
        for (int l = 0; l < kChunk; ++l)
          if (l < un.y) {
            Z rr = sk == 0 ? acc[l] : sk == 1 ? make_neg(acc[l]) : cmul(sc, acc[l]);
            if (g.accumulate) rr = cadd(yc[(long long)l * g.ys_v], rr);
            yc[(long long)l * g.ys_v] = rr;
          }
      }
    }
  }
}

template <typename Z>
static void bd_mult2_t(const BdGeom& g, const Z* X, Z* Y, const Z* M, const BdItem* items, long long nitems,
                       const int* nunits, const int4* units, const long long* udoff, int ustride, int max_units,
                       cudaStream_t st) {
  if (nitems <= 0) return;
  const long long E = g.left ? (long long)g.U * max_units * g.Wd : (long long)g.U * g.Vd * max_units;
  unsigned bx = grid_for(E, 256, 4096);
  long long by = 65535;
  long long want = (8192 + bx - 1) / bx;
  if (want < by) by = want;
  if (by > nitems) by = nitems;
  if (by < 1) by = 1;
  k_bd_mult2<Z><<<dim3(bx, (unsigned)by), 256, 0, st>>>(g, X, Y, M, items, nitems, nunits, units, udoff, ustride);
}
void bd_mult2(const BdGeom& g, const double2* X, double2* Y, const double2* M, const BdItem* items, long long nitems,
              const int* nunits, const int4* units, const long long* udoff, int ustride, int max_units,
              cudaStream_t st) {
  bd_mult2_t<double2>(g, X, Y, M, items, nitems, nunits, units, udoff, ustride, max_units, st);
}
void bd_mult2(const BdGeom& g, const float2* X, float2* Y, const float2* M, const BdItem* items, long long nitems,
              const int* nunits, const int4* units, const long long* udoff, int ustride, int max_units,
              cudaStream_t st) {
  bd_mult2_t<float2>(g, X, Y, M, items, nitems, nunits, units, udoff, ustride, max_units, st);
}

// ---------------------------------------------------------------------------
// Block Gram products with long K:  out[m][n] = alpha sum_r sum_k A_r[m][k] conj(B_r[n][k]).
// Each unit covers one <= 32x32 tile of one output block and a range of
// pairs r; it writes its partial sums, and gram_reduce adds the partials of
// a tile in a fixed order (deterministic).  Small tiles split K across the
// threads so that every lane does useful multiply-adds.
// ---------------------------------------------------------------------------
constexpr int kGramSlots = 544;  // per operand: rows x (chunk + 1) complex, see chunk_for()

__device__ __forceinline__ int gram_chunk(int rows) {
  // shared tile holds rows x chunk elements, 512 per operand
  return rows <= 1 ? 512 : rows <= 2 ? 256 : rows <= 4 ? 128 : rows <= 8 ? 64 : rows <= 16 ? 32 : 16;
}

template <typename Z>
__global__ void __launch_bounds__(256) k_gram_partials(GramGeom g, const Z* __restrict__ A,
                                                       const Z* __restrict__ B,
                                                       const GramUnit* __restrict__ units,
                                                       Z* __restrict__ partial) {
  __shared__ Z As[kGramSlots];
  __shared__ Z Bs[kGramSlots];
  __shared__ Z red[256];
  const GramUnit u = units[blockIdx.x];
  const int tid = threadIdx.x;
  const int rmax = u.rows_m > u.rows_n ? u.rows_m : u.rows_n;
  const int KC = gram_chunk(rmax);
  const int LD = KC + 1;
  const bool tri = u.tri != 0;  // square diagonal tile of a Hermitian block: elements i <= j only
  const int mn = tri ? u.rows_m * (u.rows_m + 1) / 2 : u.rows_m * u.rows_n;
  // Every lane works on a real output: up to 4 outputs per thread for large tiles,
  // K split over P phases for small ones.  No padded rows are ever multiplied.
  const int P = mn >= 256 ? 1 : 256 / mn;
  const int kp = tid / (mn < 256 ? mn : 256);
  const int nown = mn >= 256 ? (mn - tid + 255) / 256 : (kp < P ? 1 : 0);
  int em[4], en[4];
#pragma unroll
  for (int i = 0; i < 4; ++i) {
    int e = (mn >= 256 ? tid + 256 * i : tid % mn);
    if (tri) {
      // row-major upper triangle: row r holds rows_m - r elements
      int r = 0;
      while (r < u.rows_m - 1 && e >= u.rows_m - r) {
        e -= u.rows_m - r;
        ++r;
      }
      em[i] = r;
      en[i] = r + e < u.rows_m ? r + e : u.rows_m - 1;
    } else {
      em[i] = e / u.rows_n;
      en[i] = e - em[i] * u.rows_n;
    }
  }
  Z acc[4];
#pragma unroll
  for (int i = 0; i < 4; ++i) acc[i] = czero<Z>();
  const int K = g.k_inner * g.k_outer;
  for (int r = u.r0; r < u.r1; ++r) {
    const Z* Ap = A + u.a_off + (long long)(r - u.r0) * g.a_pair;
    const Z* Bp = B + u.b_off + (long long)(r - u.r0) * g.b_pair;
    for (int k0 = 0; k0 < K; k0 += KC) {
      for (int idx = tid; idx < rmax * KC; idx += 256) {
        const int i = idx / KC, kk = idx - i * KC;
        const int k = k0 + kk;
        if (k < K) {
          const int ko = k / g.k_inner, ki = k - ko * g.k_inner;
          if (i < u.rows_m) As[i * LD + kk] = Ap[(long long)i * g.a_row + (long long)ko * g.k_outer_a + ki];
          if (i < u.rows_n) Bs[i * LD + kk] = Bp[(long long)i * g.b_row + (long long)ko * g.k_outer_b + ki];
        } else {
          if (i < u.rows_m) As[i * LD + kk] = czero<Z>();
          if (i < u.rows_n) Bs[i * LD + kk] = czero<Z>();
        }
      }
      __syncthreads();
      const int kend = (K - k0) < KC ? (K - k0) : KC;
      if (std::is_same<Z, float2>::value && mn >= 256 && !tri) {
        // single precision: 2x2 register tile (rows ty, ty+16; columns tx, tx+16) halves the shared loads
        const int ty = tid >> 4, tx = tid & 15;
        const bool m0 = ty < u.rows_m, m1 = ty + 16 < u.rows_m, n0 = tx < u.rows_n, n1 = tx + 16 < u.rows_n;
        for (int kk = 0; kk < kend; ++kk) {
          const Z a0 = m0 ? As[ty * LD + kk] : czero<Z>(), a1 = m1 ? As[(ty + 16) * LD + kk] : czero<Z>();
          const Z b0 = n0 ? Bs[tx * LD + kk] : czero<Z>(), b1 = n1 ? Bs[(tx + 16) * LD + kk] : czero<Z>();
          acc[0] = cfma_cj(a0, b0, acc[0]);
          acc[1] = cfma_cj(a0, b1, acc[1]);
          acc[2] = cfma_cj(a1, b0, acc[2]);
          acc[3] = cfma_cj(a1, b1, acc[3]);
        }
      } else if (mn >= 256) {
#pragma unroll
        for (int i = 0; i < 4; ++i) {
          if (i < nown) {
            const Z* ar = As + em[i] * LD;
            const Z* br = Bs + en[i] * LD;
            Z a = acc[i];
            for (int kk = 0; kk < kend; ++kk) a = cfma_cj(ar[kk], br[kk], a);
            acc[i] = a;
          }
        }
      } else if (kp < P) {
        const Z* ar = As + em[0] * LD;
        const Z* br = Bs + en[0] * LD;
        Z a = acc[0];
        for (int kk = kp; kk < kend; kk += P) a = cfma_cj(ar[kk], br[kk], a);
        acc[0] = a;
      }
      __syncthreads();
    }
  }
  Z* out = partial + (long long)u.slot * 1024;
  if (std::is_same<Z, float2>::value && mn >= 256 && !tri) {
    const int ty = tid >> 4, tx = tid & 15;
    if (ty < u.rows_m && tx < u.rows_n) out[ty * 32 + tx] = acc[0];
    if (ty < u.rows_m && tx + 16 < u.rows_n) out[ty * 32 + tx + 16] = acc[1];
    if (ty + 16 < u.rows_m && tx < u.rows_n) out[(ty + 16) * 32 + tx] = acc[2];
    if (ty + 16 < u.rows_m && tx + 16 < u.rows_n) out[(ty + 16) * 32 + tx + 16] = acc[3];
  } else if (mn >= 256) {
#pragma unroll
    for (int i = 0; i < 4; ++i)
      if (i < nown) out[em[i] * 32 + en[i]] = acc[i];
  } else {
    red[tid] = acc[0];
    __syncthreads();
    if (tid < mn) {
      Z s = czero<Z>();
      for (int p = 0; p < P; ++p) s = cadd(s, red[p * mn + tid]);
      out[em[0] * 32 + en[0]] = s;
    }
  }
}

template <typename Z>
__global__ void __launch_bounds__(256) k_gram_reduce(const GramTile* __restrict__ tiles,
                                                     const Z* __restrict__ partial, double2* __restrict__ out,
                                                     double2 alpha, int accumulate) {
  const GramTile t = tiles[blockIdx.x];
  for (int e = threadIdx.x; e < t.rows_m * t.rows_n; e += blockDim.x) {
    const int i = e / t.rows_n, j = e - i * t.rows_n;
    if (t.tri && i > j) continue;  // below the diagonal of a Hermitian block: filled by transposition
    double2 s = make_double2(0, 0);
    for (int q = 0; q < t.unit_count; ++q) {
      const Z p = partial[(long long)(t.unit_begin + q) * 1024 + i * 32 + j];
      s.x += (double)p.x;
      s.y += (double)p.y;
    }
    s = cmul(alpha, s);
    double2* o = out + t.out_off + (long long)i * t.ld + j;
    if (accumulate) s = cadd(*o, s);
    *o = s;
  }
}

void gram_partials(const GramGeom& g, const double2* A, const double2* B, const GramUnit* units, int nunits,
                   double2* partial, cudaStream_t st) {
  if (nunits <= 0) return;
  k_gram_partials<double2><<<nunits, 256, 0, st>>>(g, A, B, units, partial);
}
void gram_partials(const GramGeom& g, const float2* A, const float2* B, const GramUnit* units, int nunits,
                   float2* partial, cudaStream_t st) {
  if (nunits <= 0) return;
  k_gram_partials<float2><<<nunits, 256, 0, st>>>(g, A, B, units, partial);
}

void gram_reduce(const GramTile* tiles, int ntiles, const double2* partial, double2* out, double2 alpha, int accumulate,
                 cudaStream_t st) {
  if (ntiles <= 0) return;
  k_gram_reduce<double2><<<ntiles, 256, 0, st>>>(tiles, partial, out, alpha, accumulate);
}
void gram_reduce(const GramTile* tiles, int ntiles, const float2* partial, double2* out, double2 alpha, int accumulate,
                 cudaStream_t st) {
  if (ntiles <= 0) return;
  k_gram_reduce<float2><<<ntiles, 256, 0, st>>>(tiles, partial, out, alpha, accumulate);
}

// precision conversion of packed families
__global__ void k_to_c64(const double2* __restrict__ a, float2* __restrict__ b, long long n) {
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
    b[i] = make_float2((float)a[i].x, (float)a[i].y);
}
void to_c64(const double2* a, float2* b, long long n, cudaStream_t st) {
  if (n > 0) k_to_c64<<<grid_for(n, 256, 8192), 256, 0, st>>>(a, b, n);
}

// Each block made Hermitian from its upper triangle: one CTA per block, rows over warps, columns
// over lanes (reads above the diagonal, writes below it and the diagonal's imaginary part: no
// overlap).  A Hermitian matrix has a real diagonal; leaving the rounding-level imaginary part of
// a diagonal computed from a slightly non-Hermitian operand would feed an anti-Hermitian
// component back into the self-consistency loop, which can amplify it from pass to pass.
__global__ void __launch_bounds__(256) k_hermitian_fill(const HermItem* __restrict__ items, double2* __restrict__ out) {
  const HermItem it = items[blockIdx.x];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  double2* B = out + it.off;
  for (int i = threadIdx.x; i < it.n; i += 256) B[(long long)i * it.n + i].y = 0.0;
  for (int i = warp + 1; i < it.n; i += 8)
    for (int j = lane; j < i; j += 32) {
      const double2 u = B[(long long)j * it.n + i];
      B[(long long)i * it.n + j] = make_double2(u.x, -u.y);
    }
}
void hermitian_fill(const HermItem* items, int nitems, double2* out, cudaStream_t st) {
  if (nitems > 0) k_hermitian_fill<<<nitems, 256, 0, st>>>(items, out);
}

// X <- (X + X^dagger) / 2 per block: one CTA per block; the thread of pair (i, j), i > j, reads
// and writes both elements of the pair, the diagonal keeps its real part.
__global__ void __launch_bounds__(256) k_hermitian_part(const HermItem* __restrict__ items, double2* __restrict__ X) {
  const HermItem it = items[blockIdx.x];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  double2* B = X + it.off;
  for (int i = threadIdx.x; i < it.n; i += 256) B[(long long)i * it.n + i].y = 0.0;
  for (int i = warp + 1; i < it.n; i += 8)
    for (int j = lane; j < i; j += 32) {
      const double2 lo = B[(long long)i * it.n + j], up = B[(long long)j * it.n + i];
      const double2 m = make_double2(0.5 * (up.x + lo.x), 0.5 * (up.y - lo.y));  // (up + conj(lo)) / 2
      B[(long long)j * it.n + i] = m;
      B[(long long)i * it.n + j] = make_double2(m.x, -m.y);
    }
}
void hermitian_part(const HermItem* items, int nitems, double2* X, cudaStream_t st) {
  if (nitems > 0) k_hermitian_part<<<nitems, 256, 0, st>>>(items, X);
}

// P0 past the middle tau node from its partner block at the mirrored node, in two launches over
// 32 x 32 output tiles of every block (one CTA per tile and tau value, so a large block spreads
// over many SMs):
//   step 0: T[i][c] = sum_a M[i][a] S[c][a]            (T in scratch, S = P0 at beta - tau)
//   step 1: R[i][j] = sum_c T[i][c] conj(M[j][c])     (R = P0 at tau)
// Both are C[i][j] = sum_k A[i][k] op(B[j][k]); k runs in steps of 16 through shared memory
// (A and B tiles stored k-major, padded rows); a thread holds 4 outputs of one column.
template <int STEP>
__global__ void __launch_bounds__(256) k_p0_reflect(const ReflItem* __restrict__ items,
                                                    const ReflTile* __restrict__ tiles, double2* __restrict__ P0,
                                                    long long p_elems, int nt, int h, const double2* __restrict__ M,
                                                    double2* __restrict__ scratch) {
  __shared__ double2 As[16][33], Bs[16][33];
  const ReflTile tl = tiles[blockIdx.x];
  const ReflItem it = items[tl.item];
  const int t = h + blockIdx.y, n = it.n;
  const double2* A;
  const double2* B;
  double2* C;
  if (STEP == 0) {
    A = M + it.m_off;
    B = P0 + (long long)(nt - 1 - t) * p_elems + it.src_off;
    C = scratch + (long long)blockIdx.y * p_elems + it.dst_off;
  } else {
    A = scratch + (long long)blockIdx.y * p_elems + it.dst_off;
    B = M + it.m_off;
    C = P0 + (long long)t * p_elems + it.dst_off;
  }
  const int i0 = 32 * tl.ti, j0 = 32 * tl.tj;
  const int tx = threadIdx.x & 31, ty = threadIdx.x >> 5;
  const double2 zero = make_double2(0.0, 0.0);
  double2 acc[4] = {zero, zero, zero, zero};
  for (int k0 = 0; k0 < n; k0 += 16) {
    for (int e = threadIdx.x; e < 512; e += 256) {
      const int r = e >> 4, kk = e & 15, k = k0 + kk;
      const int ia = i0 + r, jb = j0 + r;
      As[kk][r] = (ia < n && k < n) ? A[(long long)ia * n + k] : zero;
      Bs[kk][r] = (jb < n && k < n) ? B[(long long)jb * n + k] : zero;
    }
    __syncthreads();
#pragma unroll 4
    for (int kk = 0; kk < 16; ++kk) {
      double2 b = Bs[kk][tx];
      if (STEP == 1) b.y = -b.y;
#pragma unroll
      for (int r = 0; r < 4; ++r) acc[r] = cfma(As[kk][ty + 8 * r], b, acc[r]);
    }
    __syncthreads();
  }
#pragma unroll
  for (int r = 0; r < 4; ++r) {
    const int i = i0 + ty + 8 * r, j = j0 + tx;
    if (i < n && j < n) C[(long long)i * n + j] = acc[r];
  }
}
void p0_reflect(const ReflItem* items, const ReflTile* tiles, int ntiles, double2* P0, long long p_elems, int nt, int h,
                const double2* M, double2* scratch, cudaStream_t st) {
  if (ntiles <= 0 || nt <= h) return;
  const dim3 grid(ntiles, nt - h);
  k_p0_reflect<0><<<grid, 256, 0, st>>>(items, tiles, P0, p_elems, nt, h, M, scratch);
  k_p0_reflect<1><<<grid, 256, 0, st>>>(items, tiles, P0, p_elems, nt, h, M, scratch);
}

// dst = src^dagger per item: one CTA per item walks 32 x 32 tiles through shared memory (rows read
// and written along the fast index; the padded tile keeps each 8-lane phase on distinct banks).
__global__ void __launch_bounds__(256) k_block_adjoint(const AdjItem* __restrict__ items, double2* __restrict__ X) {
  __shared__ double2 tile[32][33];
  const AdjItem it = items[blockIdx.x];
  const int n = it.n;
  const double2* S = X + it.src_off;
  double2* D = X + it.dst_off;
  const int tx = threadIdx.x & 31, ty = threadIdx.x >> 5;
  for (int i0 = 0; i0 < n; i0 += 32)
    for (int j0 = 0; j0 < n; j0 += 32) {
      for (int r = ty; r < 32; r += 8) {
        const int i = i0 + r, j = j0 + tx;
        if (i < n && j < n) tile[r][tx] = S[(long long)i * n + j];
      }
      __syncthreads();
      for (int r = ty; r < 32; r += 8) {  // D[j0 + r][i0 + tx] = conj(S[i0 + tx][j0 + r])
        const int dr = j0 + r, dc = i0 + tx;
        if (dr < n && dc < n) {
          const double2 v = tile[tx][r];
          D[(long long)dr * n + dc] = make_double2(v.x, -v.y);
        }
      }
      __syncthreads();
    }
}
void block_adjoint(const AdjItem* items, int nitems, double2* X, cudaStream_t st) {
  if (nitems > 0) k_block_adjoint<<<nitems, 256, 0, st>>>(items, X);
}

// ---------------------------------------------------------------------------
// Series map along the tau / frequency axis: out[m][e] = alpha sum_t T[m][t] in[t][e].
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(256) k_series_map(const double2* __restrict__ T, int nm, int nt,
                                                    const double2* __restrict__ in, long long in_ld,
                                                    double2* __restrict__ out, long long out_ld, long long E,
                                                    double2 alpha, int accumulate) {
  for (int m = blockIdx.y; m < nm; m += gridDim.y) {
    const double2* Tm = T + (long long)m * nt;
    for (long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x; e < E; e += (long long)gridDim.x * blockDim.x) {
      double2 s = make_double2(0, 0);
      for (int t = 0; t < nt; ++t) s = cfma(Tm[t], in[(long long)t * in_ld + e], s);
      s = cmul(alpha, s);
      double2* o = out + (long long)m * out_ld + e;
      if (accumulate) s = cadd(*o, s);
      *o = s;
    }
  }
}

void series_map(const double2* T, int nm, int nt, const double2* in, long long in_ld, double2* out, long long out_ld,
                long long E, double2 alpha, int accumulate, cudaStream_t st) {
  if (nm <= 0 || E <= 0) return;
  unsigned bx = grid_for(E, 256, 2048);
  unsigned by = nm < 65535 ? nm : 65535;
  k_series_map<<<dim3(bx, by), 256, 0, st>>>(T, nm, nt, in, in_ld, out, out_ld, E, alpha, accumulate);
}

// ---------------------------------------------------------------------------
// Batched Gauss-Jordan inversion with partial pivoting.
//   INV_W          : A = I - P0(i Omega)_B          -> out = A^{-1} - I = [I - P0]^{-1} P0
//   INV_DYSON_STORE: A = (i w + mu) S - F - Sigma(i w) -> out = A^{-1} = G(i w)
//   INV_DYSON_TRACE: as above, trace_partial[item] = (Re weight Tr[G S], -Re weight Tr[G S G S])
//                    with G = A^{-1}: the item's share of N(mu) and of dN/dmu (dG/dmu = -G S G)
// Blocks of up to 32 take one warp each (k_invert_warp); larger ones one CTA of 8 warps each
// (k_invert_cta), the matrix in shared memory up to n = 90 (rows padded to an odd stride, so a
// column read by 32 threads takes the minimum number of wavefronts) and in a per-CTA slot of a
// global scratch buffer (L2-resident) above.
// ---------------------------------------------------------------------------
constexpr int kInvSmemMaxN = 90;
constexpr int kInvMaxN = 1024;  // bound of the per-CTA pivot and column arrays
constexpr int kInvScratchSlots = 304;

// CTA per block.  Step k of the elimination: (1) every thread copies column k, warp 0 finds the
// pivot row p (largest |a_ik|, i >= k); (2) rows k and p are exchanged and the new pivot row is
// scaled by 1/a_pk, its diagonal set to 1/a_pk; (3) each warp takes rows i != k, its lanes the
// columns j: a_ij <- [j != k] a_ij - c_i a_kj with c_i row i's column-k entry after the exchange.
// Rows are spread over warps and columns over lanes, so no thread divides an index.  The column
// exchanges that undo the row pivoting are applied row by row at the end (each thread walks its
// own rows through the swap sequence in reverse).
__global__ void __launch_bounds__(256) k_invert_cta(int mode, const InvItem* __restrict__ items, int nitems,
                                                    int slot_elems, const double2* __restrict__ Asrc,
                                                    const double2* __restrict__ S, const double2* __restrict__ F,
                                                    const double* __restrict__ nu, double mu_host,
                                                    const double* __restrict__ mu_dev,
                                                    const double* __restrict__ done_dev, double2* __restrict__ out,
                                                    double2* __restrict__ tpart, double2* __restrict__ scratch,
                                                    int* __restrict__ status, int use_smem) {
  if (done_dev != nullptr && *done_dev != 0.0) return;  // a finished search skips its remaining trials
  const double mu = mu_dev != nullptr ? *mu_dev : mu_host;
  extern __shared__ double2 smem[];
  __shared__ double2 col[kInvMaxN];
  __shared__ int perm[kInvMaxN];
  __shared__ int s_piv;
  __shared__ double s_red[4][8];
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  constexpr int NW = 8;
  double2* A = use_smem ? smem : scratch + (long long)blockIdx.x * slot_elems;
  for (int itx = blockIdx.x; itx < nitems; itx += gridDim.x) {
    const InvItem it = items[itx];
    const int n = it.n;
    const int ld = use_smem ? (n | 1) : n;
    // assemble
    for (int i = warp; i < n; i += NW) {
      for (int j = lane; j < n; j += 32) {
        const long long e = (long long)i * n + j;
        double2 a;
        if (mode == INV_W) {
          const double2 pv = Asrc[it.a_off + e];
          a = make_double2((i == j ? 1.0 : 0.0) - pv.x, -pv.y);
        } else {
          const double2 sv = S[it.s_off + e], fv = F[it.f_off + e], sg = Asrc[it.a_off + e];
          const double w = nu[it.m];
          a.x = mu * sv.x - w * sv.y - fv.x - sg.x;  // (i w + mu) s - f - sigma
          a.y = mu * sv.y + w * sv.x - fv.y - sg.y;
        }
        A[i * ld + j] = a;
      }
    }
    __syncthreads();
    for (int k = 0; k < n; ++k) {
      // (1) column k and the pivot
      for (int i = tid; i < n; i += blockDim.x) col[i] = A[i * ld + k];
      if (warp == 0) {
        double best = -1.0;
        int bi = k;
        for (int i = k + lane; i < n; i += 32) {
          const double v = cabs2(A[i * ld + k]);
          if (v > best) { best = v; bi = i; }
        }
        for (int off = 16; off > 0; off >>= 1) {
          const double ob = __shfl_down_sync(0xffffffffu, best, off);
          const int oi = __shfl_down_sync(0xffffffffu, bi, off);
          if (ob > best || (ob == best && oi < bi)) { best = ob; bi = oi; }
        }
        if (lane == 0) { s_piv = bi; perm[k] = bi; }
      }
      __syncthreads();
      const int p = s_piv;
      double2 piv = col[p];
      const double pm = cabs2(piv);
      if (!(pm > 1e-300)) {
        if (tid == 0) atomicExch(status, (int)DEV_SINGULAR);
        piv = make_double2(1.0, 0.0);
      }
      const double den = pm > 1e-300 ? pm : 1.0;
      const double2 inv = make_double2(piv.x / den, -piv.y / den);
      // (2) exchange rows k and p; scale the pivot row
      for (int j = tid; j < n; j += blockDim.x) {
        const double2 rk = A[k * ld + j], rp = A[p * ld + j];
        if (p != k) A[p * ld + j] = rk;
        A[k * ld + j] = (j == k) ? inv : cmul(rp, inv);
      }
      __syncthreads();
      // (3) eliminate column k from the other rows
      for (int i = warp; i < n; i += NW) {
        if (i == k) continue;
        const double2 c = (i == p) ? col[k] : col[i];
        for (int j = lane; j < n; j += 32) {
          const double2 pr = A[k * ld + j];
          const double2 base = (j == k) ? make_double2(0.0, 0.0) : A[i * ld + j];
          A[i * ld + j] = make_double2(base.x - (c.x * pr.x - c.y * pr.y), base.y - (c.x * pr.y + c.y * pr.x));
        }
      }
      __syncthreads();
    }
    // undo the pivoting on the columns, row by row
    for (int i = tid; i < n; i += blockDim.x) {
      double2* r = A + (long long)i * ld;
      for (int k = n - 1; k >= 0; --k) {
        const int pk = perm[k];
        if (pk != k) {
          const double2 t = r[k];
          r[k] = r[pk];
          r[pk] = t;
        }
      }
    }
    __syncthreads();
    if (mode == INV_W || mode == INV_DYSON_STORE) {
      for (int i = warp; i < n; i += NW)
        for (int j = lane; j < n; j += 32) {
          double2 a = A[i * ld + j];
          if (mode == INV_W && i == j) a.x -= 1.0;
          out[it.out_off + (long long)i * n + j] = a;
        }
    } else {
      // Tr[G S] and Tr[(G S)^2]: thread (i, j) forms X_ij = (G S)_ij and X_ji without storing X
      const double2* Sb = S + it.s_off;
      double2 t1 = make_double2(0.0, 0.0), t2 = make_double2(0.0, 0.0);
      for (int i = warp; i < n; i += NW)
        for (int j = lane; j < n; j += 32) {
          double2 xij = make_double2(0.0, 0.0), xji = make_double2(0.0, 0.0);
          for (int l = 0; l < n; ++l) {
            xij = cfma(A[i * ld + l], Sb[(long long)l * n + j], xij);
            xji = cfma(A[j * ld + l], Sb[(long long)l * n + i], xji);
          }
          if (i == j) t1 = cadd(t1, xij);
          t2 = cfma(xij, xji, t2);
        }
      for (int off = 16; off > 0; off >>= 1) {
        t1.x += __shfl_down_sync(0xffffffffu, t1.x, off);
        t1.y += __shfl_down_sync(0xffffffffu, t1.y, off);
        t2.x += __shfl_down_sync(0xffffffffu, t2.x, off);
        t2.y += __shfl_down_sync(0xffffffffu, t2.y, off);
      }
      if (lane == 0) {
        s_red[0][warp] = t1.x;
        s_red[1][warp] = t1.y;
        s_red[2][warp] = t2.x;
        s_red[3][warp] = t2.y;
      }
      __syncthreads();
      if (tid == 0) {
        double2 a = make_double2(0.0, 0.0), b = make_double2(0.0, 0.0);
        for (int w = 0; w < NW; ++w) {
          a.x += s_red[0][w];
          a.y += s_red[1][w];
          b.x += s_red[2][w];
          b.y += s_red[3][w];
        }
        const double2 tn = cmul(it.weight, a);
        const double2 td = cmul(it.weight, b);
        tpart[it.slot] = make_double2(tn.x, -td.x);  // (N part, dN/dmu part)
      }
    }
    __syncthreads();
  }
}

// Warp-per-matrix variant for blocks of at most 32: lane i owns row i.  Each pivot step is
// one warp-wide argmax, one row swap and one scaled-row broadcast; every lane then updates its
// own row with independent multiply-adds (no serial chain over rows).
constexpr int kWarpInvN = 32;
constexpr int kWarpInvSmemMax = 8 * kWarpInvN * (kWarpInvN + 1) * (int)sizeof(double2);  // 135168 B
__global__ void __launch_bounds__(256) k_invert_warp(int mode, const InvItem* __restrict__ items, int nitems,
                                                     const double2* __restrict__ Asrc, const double2* __restrict__ S,
                                                     const double2* __restrict__ F, const double* __restrict__ nu,
                                                     double mu_host, const double* __restrict__ mu_dev,
                                                     const double* __restrict__ done_dev, double2* __restrict__ out,
                                                     double2* __restrict__ tpart, int* __restrict__ status,
                                                     int slot_n) {
  // dynamic shared memory: one slot per warp of slot_n rows x (slot_n + 1) complex (padded rows),
  // two in the trace mode (the inverse, then X = G S)
  extern __shared__ double2 smdyn[];
  if (done_dev != nullptr && *done_dev != 0.0) return;
  const double mu = mu_dev != nullptr ? *mu_dev : mu_host;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int wpc = blockDim.x >> 5;
  const int itx = blockIdx.x * wpc + warp;
  if (itx >= nitems) return;
  const InvItem it = items[itx];
  const int n = it.n, ld = slot_n + 1;
  const int nbuf = mode == INV_DYSON_TRACE ? 2 : 1;
  double2* A = smdyn + (long long)warp * nbuf * slot_n * ld;
  for (int e = lane; e < n * n; e += 32) {
    const int i = e / n, j = e - i * n;
    double2 a;
    if (mode == INV_W) {
      const double2 p = Asrc[it.a_off + e];
      a = make_double2((i == j ? 1.0 : 0.0) - p.x, -p.y);
    } else {
      const double2 s = S[it.s_off + e], f = F[it.f_off + e], sg = Asrc[it.a_off + e];
      const double w = nu[it.m];
      a.x = mu * s.x - w * s.y - f.x - sg.x;
      a.y = mu * s.y + w * s.x - f.y - sg.y;
    }
    A[i * ld + j] = a;
  }
  __syncwarp();
  int myperm = lane;  // lane k records the row swapped into position k
  double2* row = A + lane * ld;
  for (int k = 0; k < n; ++k) {
    double best = (lane >= k && lane < n) ? cabs2(row[k]) : -1.0;
    int bi = (lane >= k && lane < n) ? lane : n;
    for (int off = 16; off > 0; off >>= 1) {
      const double ob = __shfl_down_sync(0xffffffffu, best, off);
      const int oi = __shfl_down_sync(0xffffffffu, bi, off);
      if (ob > best || (ob == best && oi < bi)) { best = ob; bi = oi; }
    }
    const int p = __shfl_sync(0xffffffffu, bi, 0);
    if (lane == k) myperm = p;
    if (p != k && lane < n) {  // lane j swaps column j of rows k and p
      const double2 t = A[k * ld + lane];
      A[k * ld + lane] = A[p * ld + lane];
      A[p * ld + lane] = t;
    }
    __syncwarp();
    double2 piv = A[k * ld + k];
    const double pm = cabs2(piv);
    if (!(pm > 1e-300)) {
      if (lane == 0) atomicExch(status, (int)DEV_SINGULAR);
      piv = make_double2(1.0, 0.0);
    }
    const double den = pm > 1e-300 ? pm : 1.0;
    const double2 inv = make_double2(piv.x / den, -piv.y / den);
    const double2 c = lane < n ? row[k] : make_double2(0.0, 0.0);  // multiplier of my row
    __syncwarp();
    if (lane < n) A[k * ld + lane] = (lane == k) ? inv : cmul(A[k * ld + lane], inv);  // scaled pivot row
    __syncwarp();
    if (lane < n && lane != k) {
      const double2* pr = A + k * ld;
      for (int j = 0; j < n; ++j) {
        if (j == k) {
          const double2 t = cmul(c, inv);
          row[k] = make_double2(-t.x, -t.y);
        } else {
          const double2 t = cmul(c, pr[j]);
          row[j] = make_double2(row[j].x - t.x, row[j].y - t.y);
        }
      }
    }
    __syncwarp();
  }
  for (int k = n - 1; k >= 0; --k) {
    const int p = __shfl_sync(0xffffffffu, myperm, k);
    if (p != k && lane < n) {
      const double2 t = row[k];
      row[k] = row[p];
      row[p] = t;
    }
  }
  __syncwarp();
  if (mode == INV_W) {
    for (int e = lane; e < n * n; e += 32) {
      const int i = e / n, j = e - i * n;
      double2 a = A[i * ld + j];
      if (i == j) a.x -= 1.0;
      out[it.out_off + e] = a;
    }
  } else if (mode == INV_DYSON_STORE) {
    for (int e = lane; e < n * n; e += 32) {
      const int i = e / n, j = e - i * n;
      out[it.out_off + e] = A[i * ld + j];
    }
  } else {
    // lane i: row i of X = G S into the second slot, then X_ii and sum_j X_ij X_ji
    double2* X = A + slot_n * ld;
    const double2* Sb = S + it.s_off;
    if (lane < n) {
      for (int j = 0; j < n; ++j) {
        double2 x = make_double2(0.0, 0.0);
        for (int l = 0; l < n; ++l) x = cfma(row[l], Sb[l * n + j], x);
        X[lane * ld + j] = x;
      }
    }
    __syncwarp();
    double2 s = make_double2(0.0, 0.0), s2 = make_double2(0.0, 0.0);
    if (lane < n) {
      s = X[lane * ld + lane];
      for (int j = 0; j < n; ++j) s2 = cfma(X[lane * ld + j], X[j * ld + lane], s2);
    }
    for (int off = 16; off > 0; off >>= 1) {
      s.x += __shfl_down_sync(0xffffffffu, s.x, off);
      s.y += __shfl_down_sync(0xffffffffu, s.y, off);
      s2.x += __shfl_down_sync(0xffffffffu, s2.x, off);
      s2.y += __shfl_down_sync(0xffffffffu, s2.y, off);
    }
    if (lane == 0) {
      const double2 t = cmul(it.weight, s);
      const double2 d = cmul(it.weight, s2);
      tpart[it.slot] = make_double2(t.x, -d.x);  // (N part, dN/dmu part)
    }
  }
}

void invert_plan(int mode, const InvPlan& pl, const double2* A, const double2* S, const double2* F, const double* nu,
                 double mu, const double* mu_dev, const double* done_dev, double2* out, double2* trace_partial,
                 double2* scratch, int* status, cudaStream_t st) {
  static bool attr = false;
  if (!attr) {
    cudaFuncSetAttribute(k_invert_warp, cudaFuncAttributeMaxDynamicSharedMemorySize, kWarpInvSmemMax);
    cudaFuncSetAttribute(k_invert_cta, cudaFuncAttributeMaxDynamicSharedMemorySize,
                         kInvSmemMaxN * (kInvSmemMaxN | 1) * (int)sizeof(double2));
    attr = true;
  }
  const int nmid = pl.nitems - pl.nsmall - pl.nscr;
  // the three groups are independent: when two or more are present they run on the side streams
  // (when given) and share the GPU
  const int ngroups = (pl.nscr > 0) + (nmid > 0) + (pl.nsmall > 0);
  const bool fork = ngroups > 1 && pl.aux[0] != nullptr && pl.aux[1] != nullptr;
  cudaStream_t s_mid = fork ? pl.aux[0] : st, s_small = fork ? pl.aux[1] : st;
  if (fork) {
    cudaEventRecord(pl.fork, st);
    cudaStreamWaitEvent(pl.aux[0], pl.fork, 0);
    cudaStreamWaitEvent(pl.aux[1], pl.fork, 0);
  }
  if (pl.nscr > 0) {  // the largest blocks first, each in a global scratch slot
    const int grid = pl.nscr < kInvScratchSlots ? pl.nscr : kInvScratchSlots;
    k_invert_cta<<<grid, 256, 0, st>>>(mode, pl.items + pl.nsmall, pl.nscr, pl.max_n * pl.max_n, A, S, F, nu, mu,
                                       mu_dev, done_dev, out, trace_partial, scratch, status, 0);
  }
  if (nmid > 0) {
    const size_t sm = (size_t)pl.mid_n * (pl.mid_n | 1) * sizeof(double2);
    k_invert_cta<<<nmid, 256, sm, s_mid>>>(mode, pl.items + pl.nsmall + pl.nscr, nmid, 0, A, S, F, nu, mu, mu_dev,
                                           done_dev, out, trace_partial, nullptr, status, 1);
  }
  if (pl.nsmall > 0) {
    const int sn = pl.small_n < 1 ? 1 : pl.small_n;
    const size_t per_warp = (size_t)(mode == INV_DYSON_TRACE ? 2 : 1) * sn * (sn + 1) * sizeof(double2);
    const int wpc = 8 * per_warp <= (size_t)kWarpInvSmemMax ? 8 : 4;  // 4 x 2 x 32 x 33 x 16 B fits
    k_invert_warp<<<(pl.nsmall + wpc - 1) / wpc, 32 * wpc, wpc * per_warp, s_small>>>(
        mode, pl.items, pl.nsmall, A, S, F, nu, mu, mu_dev, done_dev, out, trace_partial, status, sn);
  }
  if (fork) {
    cudaEventRecord(pl.join[0], pl.aux[0]);
    cudaEventRecord(pl.join[1], pl.aux[1]);
    cudaStreamWaitEvent(st, pl.join[0], 0);
    cudaStreamWaitEvent(st, pl.join[1], 0);
  }
}

// ---------------------------------------------------------------------------
// Generalised Hermitian eigensolver H C = S C eps, one CTA per matrix.
// S^{-1/2} from a Jacobi eigendecomposition of S, Jacobi on S^{-1/2} H S^{-1/2}
// (parallel cyclic Jacobi, round-robin ordering of disjoint rotations), then
// C = S^{-1/2} Y.  Works in a per-CTA slot of global scratch (3 n x n).
// ---------------------------------------------------------------------------
__device__ void jacobi_inplace(double2* A, double2* V, int n, double2* rot /* 3 * (n/2+1) */) {
  const int tid = threadIdx.x;
  const int n2 = n + (n & 1);
  for (int e = tid; e < n * n; e += blockDim.x) V[e] = make_double2((e / n) == (e % n) ? 1.0 : 0.0, 0.0);
  __syncthreads();
  __shared__ double s_off, s_tot;
  for (int sweep = 0; sweep < 60; ++sweep) {
    if (tid == 0) { s_off = 0.0; s_tot = 0.0; }
    __syncthreads();
    double off = 0.0, tot = 0.0;
    for (int e = tid; e < n * n; e += blockDim.x) {
      const double v = cabs2(A[e]);
      tot += v;
      if ((e / n) != (e % n)) off += v;
    }
    atomicAdd(&s_off, off);
    atomicAdd(&s_tot, tot);
    __syncthreads();
    const bool done = !(s_off > 1e-30 * s_tot) || s_tot == 0.0;
    __syncthreads();
    if (done) break;
    for (int round = 0; round < n2 - 1; ++round) {
      // pair i: slots i and n2-1-i; slot 0 holds player 0, slot j>0 holds ((j-1+round) mod (n2-1)) + 1
      for (int i = tid; i < n2 / 2; i += blockDim.x) {
        const int sa = i, sb = n2 - 1 - i;
        int pa = sa == 0 ? 0 : ((sa - 1 + round) % (n2 - 1)) + 1;
        int pb = ((sb - 1 + round) % (n2 - 1)) + 1;
        if (pa > pb) { const int t = pa; pa = pb; pb = t; }
        double c = 1.0, s = 0.0;
        double2 z = make_double2(1.0, 0.0);
        if (pb < n) {
          const double2 apq = A[pa * n + pb];
          const double b = sqrt(cabs2(apq));
          if (b > 1e-300) {
            z = make_double2(apq.x / b, apq.y / b);
            const double app = A[pa * n + pa].x, aqq = A[pb * n + pb].x;
            const double tau = (aqq - app) / (2.0 * b);
            const double t = (tau >= 0 ? 1.0 : -1.0) / (fabs(tau) + sqrt(1.0 + tau * tau));
            c = 1.0 / sqrt(1.0 + t * t);
            s = t * c;
          }
        }
        rot[3 * i] = make_double2(c, s);
        rot[3 * i + 1] = z;
        rot[3 * i + 2] = make_double2((double)pa, (double)pb);
      }
      __syncthreads();
      // rows: A[p,:] = c A[p,:] - s z A[q,:];  A[q,:] = s A[p,:] + c z A[q,:]
      for (int e = tid; e < (n2 / 2) * n; e += blockDim.x) {
        const int i = e / n, j = e - i * n;
        const double2 cs = rot[3 * i], z = rot[3 * i + 1];
        const int pa = (int)rot[3 * i + 2].x, pb = (int)rot[3 * i + 2].y;
        if (pb >= n || cs.y == 0.0) continue;
        const double2 ap = A[pa * n + j], aq = A[pb * n + j];
        const double2 zq = cmul(z, aq);
        A[pa * n + j] = make_double2(cs.x * ap.x - cs.y * zq.x, cs.x * ap.y - cs.y * zq.y);
        A[pb * n + j] = make_double2(cs.y * ap.x + cs.x * zq.x, cs.y * ap.y + cs.x * zq.y);
      }
      __syncthreads();
      // columns (and V): X[:,p] = c X[:,p] - s conj(z) X[:,q];  X[:,q] = s X[:,p] + c conj(z) X[:,q]
      for (int e = tid; e < (n2 / 2) * n; e += blockDim.x) {
        const int i = e / n, r = e - i * n;
        const double2 cs = rot[3 * i], z = rot[3 * i + 1];
        const int pa = (int)rot[3 * i + 2].x, pb = (int)rot[3 * i + 2].y;
        if (pb >= n || cs.y == 0.0) continue;
        const double2 zc = cconj(z);
        {
          const double2 xp = A[r * n + pa], xq = cmul(zc, A[r * n + pb]);
          A[r * n + pa] = make_double2(cs.x * xp.x - cs.y * xq.x, cs.x * xp.y - cs.y * xq.y);
          A[r * n + pb] = make_double2(cs.y * xp.x + cs.x * xq.x, cs.y * xp.y + cs.x * xq.y);
        }
        {
          const double2 xp = V[r * n + pa], xq = cmul(zc, V[r * n + pb]);
          V[r * n + pa] = make_double2(cs.x * xp.x - cs.y * xq.x, cs.x * xp.y - cs.y * xq.y);
          V[r * n + pb] = make_double2(cs.y * xp.x + cs.x * xq.x, cs.y * xp.y + cs.x * xq.y);
        }
      }
      __syncthreads();
    }
  }
}

__global__ void __launch_bounds__(256) k_geneig(const EigItem* __restrict__ items, int nitems, int max_n,
                                                const double2* __restrict__ H, const double2* __restrict__ S,
                                                double2* __restrict__ C, double* __restrict__ eps,
                                                double2* __restrict__ scratch) {
  __shared__ double2 rot[3 * 320];
  const int tid = threadIdx.x;
  const long long slot = (long long)max_n * max_n;
  double2* A = scratch + (long long)blockIdx.x * 4 * slot;
  double2* Vv = A + slot;
  double2* Sm = Vv + slot;
  double2* T = Sm + slot;
  for (int itx = blockIdx.x; itx < nitems; itx += gridDim.x) {
    const EigItem it = items[itx];
    const int n = it.n, nn = n * n;
    if (S != nullptr) {
      for (int e = tid; e < nn; e += blockDim.x) A[e] = S[it.s_off + e];
      __syncthreads();
      jacobi_inplace(A, Vv, n, rot);
      // Sm = V diag(sigma^-1/2) V^dagger
      for (int e = tid; e < nn; e += blockDim.x) {
        const int i = e / n, j = e - i * n;
        double2 s = make_double2(0, 0);
        for (int l = 0; l < n; ++l) {
          const double w = 1.0 / sqrt(A[l * n + l].x);
          const double2 t = cmul(Vv[i * n + l], cconj(Vv[j * n + l]));
          s.x += w * t.x;
          s.y += w * t.y;
        }
        Sm[e] = s;
      }
      __syncthreads();
      // T = H Sm;  A = Sm T
      for (int e = tid; e < nn; e += blockDim.x) {
        const int i = e / n, j = e - i * n;
        double2 s = make_double2(0, 0);
        for (int l = 0; l < n; ++l) s = cfma(H[it.h_off + i * n + l], Sm[l * n + j], s);
        T[e] = s;
      }
      __syncthreads();
      for (int e = tid; e < nn; e += blockDim.x) {
        const int i = e / n, j = e - i * n;
        double2 s = make_double2(0, 0);
        for (int l = 0; l < n; ++l) s = cfma(Sm[i * n + l], T[l * n + j], s);
        A[e] = s;
      }
      __syncthreads();
      for (int e = tid; e < nn; e += blockDim.x) {  // exact Hermitian symmetrisation
        const int i = e / n, j = e - i * n;
        if (i < j) {
          const double2 a = A[e], b = A[j * n + i];
          const double2 h = make_double2(0.5 * (a.x + b.x), 0.5 * (a.y - b.y));
          A[e] = h;
          A[j * n + i] = cconj(h);
        } else if (i == j) {
          A[e].y = 0.0;
        }
      }
      __syncthreads();
    } else {
      for (int e = tid; e < nn; e += blockDim.x) A[e] = H[it.h_off + e];
      __syncthreads();
    }
    jacobi_inplace(A, Vv, n, rot);
    // C = Sm V (or V), eigenvalues = diag(A) (unsorted; callers need no order)
    for (int e = tid; e < nn; e += blockDim.x) {
      const int i = e / n, j = e - i * n;
      double2 s;
      if (S != nullptr) {
        s = make_double2(0, 0);
        for (int l = 0; l < n; ++l) s = cfma(Sm[i * n + l], Vv[l * n + j], s);
      } else {
        s = Vv[e];
      }
      C[it.c_off + e] = s;
    }
    for (int i = tid; i < n; i += blockDim.x) eps[it.e_off + i] = A[i * n + i].x;
    __syncthreads();
  }
}

void geneig(const EigItem* items, int nitems, int max_n, const double2* H, const double2* S, double2* C, double* eps,
            double2* scratch, cudaStream_t st) {
  if (nitems <= 0) return;
  int grid = nitems < 304 ? nitems : 304;
  k_geneig<<<grid, 256, 0, st>>>(items, nitems, max_n, H, S, C, eps, scratch);
}

// ---------------------------------------------------------------------------
// Weighted block trace products, deterministic two-stage reduction.
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(256) k_trace_items(const TrItem* __restrict__ items, const double2* __restrict__ X,
                                                     const double2* __restrict__ Y, double2* __restrict__ partial) {
  __shared__ double2 red[256];
  const TrItem it = items[blockIdx.x];
  const int n = it.n;
  double2 s = make_double2(0, 0);
  for (int e = threadIdx.x; e < n * n; e += blockDim.x) {
    const int a = e / n, b = e - a * n;
    s = cfma(X[it.x_off + e], Y[it.y_off + (long long)b * n + a], s);
  }
  red[threadIdx.x] = s;
  __syncthreads();
  for (int off = 128; off > 0; off >>= 1) {
    if (threadIdx.x < off) red[threadIdx.x] = cadd(red[threadIdx.x], red[threadIdx.x + off]);
    __syncthreads();
  }
  if (threadIdx.x == 0) partial[blockIdx.x] = cmul(it.w, red[0]);
}

__global__ void k_sum_partials(const double2* __restrict__ partial, int n, double2* __restrict__ result) {
  __shared__ double2 red[256];
  double2 s = make_double2(0, 0);
  // fixed assignment: thread t sums t, t+256, ...; then a fixed tree
  for (int i = threadIdx.x; i < n; i += 256) s = cadd(s, partial[i]);
  red[threadIdx.x] = s;
  __syncthreads();
  for (int off = 128; off > 0; off >>= 1) {
    if (threadIdx.x < off) red[threadIdx.x] = cadd(red[threadIdx.x], red[threadIdx.x + off]);
    __syncthreads();
  }
  if (threadIdx.x == 0) *result = red[0];
}

void trace_products(const TrItem* items, int nitems, const double2* X, const double2* Y, double2* partial,
                    double2* result, cudaStream_t st) {
  if (nitems > 0) k_trace_items<<<nitems, 256, 0, st>>>(items, X, Y, partial);
  k_sum_partials<<<1, 256, 0, st>>>(partial, nitems, result);
}
void sum_partials(const double2* partial, int n, double2* result, cudaStream_t st) {
  k_sum_partials<<<1, 256, 0, st>>>(partial, n, result);
}

// ---------------------------------------------------------------------------
// small helpers
// ---------------------------------------------------------------------------
__global__ void k_fill_zero(double2* p, long long n) {
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
    p[i] = make_double2(0, 0);
}
void fill_zero(double2* p, long long n, cudaStream_t st) {
  if (n > 0) k_fill_zero<<<grid_for(n, 256, 8192), 256, 0, st>>>(p, n);
}

__global__ void k_axpby(double2* y, const double2* x, long long n, double a, double b) {
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
    const double2 yy = y[i], xx = x[i];
    y[i] = make_double2(a * yy.x + b * xx.x, a * yy.y + b * xx.y);
  }
}
void axpby(double2* y, const double2* x, long long n, double a, double b, cudaStream_t st) {
  if (n > 0) k_axpby<<<grid_for(n, 256, 8192), 256, 0, st>>>(y, x, n, a, b);
}

__global__ void k_max_abs_diff(const double2* a, const double2* b, long long n, unsigned long long* out) {
  double m = 0.0;
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
    const double dx = a[i].x - b[i].x, dy = a[i].y - b[i].y;
    const double v = sqrt(dx * dx + dy * dy);
    if (v > m) m = v;
  }
  for (int off = 16; off > 0; off >>= 1) {
    const double o = __shfl_down_sync(0xffffffffu, m, off);
    if (o > m) m = o;
  }
  if ((threadIdx.x & 31) == 0) atomicMax(out, (unsigned long long)__double_as_longlong(m));
}
void max_abs_diff(const double2* a, const double2* b, long long n, unsigned long long* out_bits, cudaStream_t st) {
  cudaMemsetAsync(out_bits, 0, sizeof(unsigned long long), st);
  if (n > 0) k_max_abs_diff<<<grid_for(n, 256, 4096), 256, 0, st>>>(a, b, n, out_bits);
}

// dense[n x n] matrices <-> packed diagonal blocks.  Block b: dense offset of
// its (0,0) element, size, packed offset; to_packed = 1 copies dense -> packed.
__global__ void k_pack_blocks(const double2* dense, double2* packed, long long dense_ld_mat, int n,
                              const long long* __restrict__ bdo, const int* __restrict__ bn,
                              const long long* __restrict__ bpo, int nblk, int to_packed) {
  double2* dd = const_cast<double2*>(dense);
  for (int b = blockIdx.y; b < nblk; b += gridDim.y) {
    const int nb = bn[b];
    for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < nb * nb; e += gridDim.x * blockDim.x) {
      const int i = e / nb, j = e - i * nb;
      const long long d = bdo[b] + (long long)i * n + j;
      if (to_packed)
        packed[bpo[b] + e] = dd[d];
      else
        dd[d] = packed[bpo[b] + e];
    }
  }
  (void)dense_ld_mat;
}
void pack_blocks(const double2* dense, long long dense_ld_mat, int n, const long long* blk_dense_off, const int* blk_n,
                 const long long* blk_pack_off, int nblk, double2* packed, int to_packed, cudaStream_t st) {
  if (nblk <= 0) return;
  unsigned by = nblk < 65535 ? nblk : 65535;
  k_pack_blocks<<<dim3(4, by), 256, 0, st>>>(dense, packed, dense_ld_mat, n, blk_dense_off, blk_n, blk_pack_off, nblk,
                                             to_packed);
}

// G0(tau) of one block from its eigenpairs: G = -C diag(g(tau)) C^dagger,
// g(tau) = exp(-xi tau) / (1 + exp(-beta xi)) written without overflow.
__global__ void k_g0(const double2* __restrict__ C, const double* __restrict__ eps,
                     const long long* __restrict__ row_boff, const int* __restrict__ row_bn,
                     const long long* __restrict__ row_eoff, long long g_elems, const double* __restrict__ tau,
                     int ntau, double beta, double mu, double2* __restrict__ G) {
  const long long total = g_elems * ntau;
  for (long long idx = (long long)blockIdx.x * blockDim.x + threadIdx.x; idx < total;
       idx += (long long)gridDim.x * blockDim.x) {
    const int t = (int)(idx / g_elems);
    const long long e = idx - (long long)t * g_elems;
    const long long boff = row_boff[e];
    const int n = row_bn[e];
    const long long eo = row_eoff[e];
    const int a = (int)((e - boff) / n), b = (int)((e - boff) % n);
    const double tt = tau[t];
    double2 s = make_double2(0, 0);
    for (int l = 0; l < n; ++l) {
      const double xi = eps[eo + l] - mu;
      double g;
      if (xi >= 0)
        g = exp(-xi * tt) / (1.0 + exp(-beta * xi));
      else
        g = exp(xi * (beta - tt)) / (exp(beta * xi) + 1.0);
      const double2 t2 = cmul(C[boff + (long long)a * n + l], cconj(C[boff + (long long)b * n + l]));
      s.x -= g * t2.x;
      s.y -= g * t2.y;
    }
    G[(long long)t * g_elems + e] = s;
  }
}
void g0_closed_form(const double2* C, const double* eps, const long long* row_boff, const int* row_bn,
                    const long long* row_eoff, long long g_elems, const double* tau, int ntau, double beta, double mu,
                    double2* G, cudaStream_t st) {
  k_g0<<<grid_for(g_elems * ntau, 256, 8192), 256, 0, st>>>(C, eps, row_boff, row_bn, row_eoff, g_elems, tau, ntau,
                                                              beta, mu, G);
}

// Chemical-potential search on the device (bracketed Newton).  State s[0] lo, s[1] hi, s[2] mu
// (the next trial, then the result), s[3] done, s[4] N of the last trial, s[5] |N - target| of
// the previous trial, s[16] running count of evaluated trials.  k_mu_start: the first trial is the start point when it lies inside
// (lo, hi), else the midpoint.  k_mu_update: sums the trial's partials (N, dN/dmu) in a fixed
// order and either stops (|N - target| <= tol) or shrinks the bracket to the side holding the
// root and picks the next trial: the Newton point mu - (N - target) / N' when N' > 0, the point
// lies strictly inside the bracket and |N - target| fell to at most half its previous value,
// else the midpoint of the bracket.
__global__ void k_mu_start(double* s, double start_host, const double* start_dev, double lo, double hi) {
  if (threadIdx.x != 0 || blockIdx.x != 0) return;
  const double m = start_dev != nullptr ? *start_dev : start_host;
  s[0] = lo;
  s[1] = hi;
  s[2] = (m > lo && m < hi) ? m : 0.5 * (lo + hi);
  s[3] = 0.0;
  s[4] = 0.0;
  s[5] = INFINITY;
}
__global__ void __launch_bounds__(256) k_mu_update(double* s, const double2* __restrict__ partial, int n,
                                                   double target, double tol) {
  if (s[3] != 0.0) return;
  __shared__ double2 red[256];
  double2 a = make_double2(0, 0);
  for (int i = threadIdx.x; i < n; i += 256) a = cadd(a, partial[i]);
  red[threadIdx.x] = a;
  __syncthreads();
  for (int off = 128; off > 0; off >>= 1) {
    if (threadIdx.x < off) red[threadIdx.x] = cadd(red[threadIdx.x], red[threadIdx.x + off]);
    __syncthreads();
  }
  if (threadIdx.x != 0) return;
  const double nn = red[0].x, dn = red[0].y, mu = s[2];
  const double r = nn - target;
  s[4] = nn;
  s[16] += 1.0;  // trials evaluated since the context was made (for flop accounting)
  if (fabs(r) <= tol) {
    s[3] = 1.0;
    return;
  }
  if (r > 0) s[1] = mu;
  else s[0] = mu;
  const double lo = s[0], hi = s[1];
  const double newton = dn > 0 ? mu - r / dn : NAN;
  s[2] = (newton > lo && newton < hi && fabs(r) <= 0.5 * s[5]) ? newton : 0.5 * (lo + hi);
  s[5] = fabs(r);
}
void mu_start(double* s, double start_host, const double* start_dev, double lo, double hi, cudaStream_t st) {
  k_mu_start<<<1, 32, 0, st>>>(s, start_host, start_dev, lo, hi);
}
void mu_update(double* s, const double2* partial, int n, double target, double tol, cudaStream_t st) {
  k_mu_update<<<1, 256, 0, st>>>(s, partial, n, target, tol);
}

// mu by bisection on (sum_i w_i f(eps_i - mu)) = target, one CTA, fixed 200 halvings.
__global__ void k_mu_bisect(const double* __restrict__ eps, const double* __restrict__ wts, int n, double beta,
                            double target, double lo, double hi, double* out) {
  __shared__ double red[256];
  __shared__ double s_lo, s_hi;
  if (threadIdx.x == 0) { s_lo = lo; s_hi = hi; }
  __syncthreads();
  for (int it = 0; it < 200; ++it) {
    const double mid = 0.5 * (s_lo + s_hi);
    double s = 0.0;
    for (int i = threadIdx.x; i < n; i += 256) {
      const double x = beta * (eps[i] - mid);
      const double f = x > 0 ? exp(-x) / (1.0 + exp(-x)) : 1.0 / (1.0 + exp(x));
      s += wts[i] * f;
    }
    red[threadIdx.x] = s;
    __syncthreads();
    for (int off = 128; off > 0; off >>= 1) {
      if (threadIdx.x < off) red[threadIdx.x] += red[threadIdx.x + off];
      __syncthreads();
    }
    if (threadIdx.x == 0) {
      if (red[0] > target) s_hi = mid; else s_lo = mid;
    }
    __syncthreads();
    if (s_hi - s_lo < 1e-13) break;
  }
  if (threadIdx.x == 0) *out = 0.5 * (s_lo + s_hi);
}
double mu_bisect_device(const double* eps, const double* wts, int n, double beta, double n_target, double lo, double hi,
                        double* work, cudaStream_t st) {
  k_mu_bisect<<<1, 256, 0, st>>>(eps, wts, n, beta, n_target, lo, hi, work);
  double mu = 0;
  cudaMemcpyAsync(&mu, work, sizeof(double), cudaMemcpyDeviceToHost, st);
  cudaStreamSynchronize(st);
  return mu;
}

}  // namespace sgw
