// Tensor-core path of the chosen form: the V-G-V chain of P0 (Eq. (P0), Algorithm 3) and the
// V-G-P-V chain of Sigma (Eq. (sigma), Algorithm 4) as grouped tcgen05 GEMMs.
//
// Every complex contraction is written as two real contractions over the interleaved (re, im)
// index of complex64 operands: for D = A B^T,
//     Re D = sum_k A[2k] (Re B) + A[2k+1] (-Im B),   Im D = sum_k A[2k] (Im B) + A[2k+1] (Re B),
// and for the Gram form D = A B^H the B factors are (Re B, Im B) and (-Im B, Re B).  The two
// B variants are built by small preparation kernels where B is a G or P block (and stays in L2),
// and inside the CTA from a single copy where B is the interaction tensor.  Each real operand
// x is carried as a TF32 head h = rn(x) and a TF32 tail l = rn(x - h) (h + l = x to about
// 2^-22); three TF32 products h*h + h*l + l*h accumulate in FP32 in tensor memory, which keeps
// the product to about FP32 accuracy.  Sums over long contraction ranges are split into units whose
// FP32 partial tiles are added in FP64 in a fixed order.
//
// One CTA = one 128-row output tile: warp 0 issues TMA loads (64-byte swizzled 32-row boxes of
// 16 reals), warp 1 owns the tensor-memory allocation and issues the MMAs, warps 2-5 split the
// staged operands into head and tail and, at the end, read the accumulators and store.  Every
// wait is bounded in time; a CTA that runs out of time records SGW status "timeout", drains its
// copies in flight, frees its tensor memory and returns.
#include <cuda.h>
#include <cudaTypedefs.h>

#include <algorithm>
#include <cmath>
#include <cstdlib>
#include <cstring>
#include <mutex>
#include <string>
#include <tuple>
#include <utility>
#include <vector>

#include "sgw_internal.h"

using namespace sgw;

namespace sgw {

// One job: an A slab range and a B operand; the CTA picks its 128-row tile of the job by blockIdx.
struct alignas(16) TcJob {
  int a_y = 0, a_z = 0, b_y = 0, b_z = 0;  // first row and slab of the A and B boxes
  int a_x = 0, b_x = 0;    // first contracted coordinate (reals, multiple of 4)
  int nslab = 1, nchunk = 1;  // contraction loop: nslab slabs x nchunk chunks of 16 reals
  int a_dz = 0, b_dz = 0;  // slab increments
  int m_rows = 0;          // rows of A the job covers (tiles of 128)
  int n_valid = 0, n_mma = 16;  // stored columns; MMA width (multiple of 16, <= 128)
  // row groups (tau stacking): g_count groups of g_rows tile rows, group g read from slab
  // a_z + g g_dz, g_valid rows of each stored; g_count = 1: one group of m_rows rows
  int g_count = 1, g_rows = 0, g_valid = 0, g_dz = 0;
  int pad0 = 0, pad1 = 0, pad2 = 0;
  long long out_off = 0;   // partial slot (Gram) or output base (affine store)
};
static_assert(sizeof(TcJob) == 96, "TcJob layout");

// Output tile of a Gram reduction over the partial tiles of its units (FP64 sum in order).
struct alignas(16) TcTile {
  long long out_off;
  int ld, m_valid, n_valid, pm0, pn0, unit_begin, unit_count, unit_stride;
};

struct TcArgs {
  int mtiles;          // 128-row tiles per job
  int a_box;           // rows per A box of the A tensor map (8 or 32)
  int mode;            // 0: FP32 partial tile [n][m] at out_off; 1: affine store
  long long Rs, S1, S2;  // affine store: out[out_off + (R / Rs) S1 + (R % Rs) + n S2], R = tile row
  float2 alpha;
  float2* out;
};

// Cached jobs of the tensor-core chains.
struct TcPlan {
  bool built_p0 = false, built_sigma = false;
  int nc_p0 = 0, nc_s = 0;
  std::vector<long long> vg_start, gvg_start, pg_start, pr_start;            // per tau: first job / unit / tile
  std::vector<long long> svg_start, pvg_start, sg_start, sr_start;
  TcJob *d_vg = nullptr, *d_gvg = nullptr, *d_pg = nullptr, *d_svg = nullptr, *d_pvg = nullptr, *d_sg = nullptr;
  TcTile *d_pr = nullptr, *d_sr = nullptr;
  long long max_units_p0 = 0, max_units_s = 0;
  bool drain_s = true;   // Sigma Gram with drained accumulators (nao <= 64)
  long long slot_s = 0;  // partial slot (complex elements) of the Sigma Gram
  int mt_vg = 0, mt_svg = 0, mt_pvg = 0;
  // block tables of the orbital partition (dense G builder) and of the auxiliary blocks (P^T builder)
  int *d_ao_start = nullptr, *d_ao_size = nullptr;
  long long* d_ao_doff = nullptr;
  long long* d_g_off = nullptr;
  int* d_ab_info = nullptr;  // per aux block: start, size, delta
  long long* d_ab_off = nullptr;
  int pt_rows = 0, pt_k = 0, ninst = 0;
  double fl_vg = 0, fl_gvg = 0, fl_pg = 0, fl_svg = 0, fl_pvg = 0, fl_sg = 0;  // algorithmic flops per tau
};

}  // namespace sgw

namespace {

constexpr int kThreads = 192;
constexpr int kTileBytes = 128 * 64;         // 128 rows x 16 fp32 (one swizzle row each)
constexpr int kStageBytes = 6 * kTileBytes;  // A head, A tail, B1 head, B1 tail, B2 head, B2 tail
constexpr int smem_bytes(int stages) { return stages * kStageBytes + 1024; }
constexpr uint32_t kTmemCols = 256;          // Re accumulator in columns [0,128), Im in [128,256)
constexpr unsigned long long kWaitNs = 2000000000ULL;  // 2 s
constexpr int kSlot = 128 * 128;             // complex elements of one partial tile (N <= 128)
constexpr int kSlotD = 128 * 64;             // same, drained kernels (N <= 64)

__device__ __forceinline__ uint32_t su32(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }
__device__ __forceinline__ unsigned long long gtime() {
  unsigned long long t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}
__device__ __forceinline__ void mbar_init(uint32_t bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(bar), "r"(count) : "memory");
}
__device__ __forceinline__ void mbar_expect_tx(uint32_t bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(bar), "r"(bytes) : "memory");
}
__device__ __forceinline__ void mbar_arrive(uint32_t bar) {
  asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(bar) : "memory");
}
__device__ __forceinline__ bool mbar_try(uint32_t bar, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n.reg .pred p;\nmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\nselp.u32 %0, 1, 0, p;\n}"
      : "=r"(ok)
      : "r"(bar), "r"(parity)
      : "memory");
  return ok != 0;
}
// Wait for the phase of the given parity; false after kWaitNs (sets *abort) or once *abort is set
// by another role (if honour_abort).
__device__ bool mbar_wait(uint32_t bar, uint32_t parity, volatile int* abort, bool honour_abort = true) {
  if (mbar_try(bar, parity)) return true;
  const unsigned long long t0 = gtime();
  while (true) {
    if (mbar_try(bar, parity)) return true;
    if (honour_abort && *abort) return false;
    if (gtime() - t0 > kWaitNs) {
      *abort = 1;
      return false;
    }
  }
}
__device__ __forceinline__ void tma_load3(uint32_t dst, const CUtensorMap* map, int x, int y, int z, uint32_t bar) {
  asm volatile(
      "cp.async.bulk.tensor.3d.shared::cluster.global.tile.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3, %4}], "
      "[%5];" ::"r"(dst),
      "l"(reinterpret_cast<uint64_t>(map)), "r"(x), "r"(y), "r"(z), "r"(bar)
      : "memory");
}
__device__ __forceinline__ void tc_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void tc_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }
// Shared-memory matrix descriptor: K-major, 64-byte swizzle, 8-row groups 512 bytes apart.
__device__ __forceinline__ uint64_t sw64_desc(uint32_t saddr) {
  return (uint64_t)((saddr & 0x3FFFFu) >> 4) | ((uint64_t)1 << 16) | ((uint64_t)(512 >> 4) << 32) |
         ((uint64_t)1 << 46) | ((uint64_t)4 << 61);
}
// Instruction descriptor: kind::tf32, FP32 accumulator, both operands K-major, M = 128.
__device__ __forceinline__ uint32_t tf32_idesc(int n) {
  return (1u << 4) | (2u << 7) | (2u << 10) | ((uint32_t)(n >> 3) << 17) | ((uint32_t)(128 >> 4) << 24);
}
__device__ __forceinline__ void umma_tf32(uint32_t d, uint64_t a, uint64_t b, uint32_t idesc, uint32_t acc) {
  asm volatile(
      "{\n.reg .pred p;\nsetp.ne.b32 p, %4, 0;\ntcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n}" ::"r"(d),
      "l"(a), "l"(b), "r"(idesc), "r"(acc)
      : "memory");
}
__device__ __forceinline__ void umma_commit(uint32_t bar) {
  asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(bar) : "memory");
}
__device__ __forceinline__ void tmem_ld16(uint32_t taddr, uint32_t* r) {
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, "
      "%15}, [%16];"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]), "=r"(r[8]),
        "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
      : "r"(taddr));
}
__device__ __forceinline__ void tmem_wait_ld() { asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory"); }

// x rounded to the nearest TF32 value (10 stored mantissa bits; the low 13 bits are zero)
__device__ __forceinline__ float tf32_rn(float x) {
  uint32_t r;
  asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(r) : "f"(x));
  return __uint_as_float(r);
}
__device__ __forceinline__ float4 head4(float4 x) {
  return make_float4(tf32_rn(x.x), tf32_rn(x.y), tf32_rn(x.z), tf32_rn(x.w));
}
// tail x - h, itself rounded to TF32: h + t = x to about 2^-22 relative
__device__ __forceinline__ float4 tail4(float4 x, float4 h) {
  return make_float4(tf32_rn(x.x - h.x), tf32_rn(x.y - h.y), tf32_rn(x.z - h.z), tf32_rn(x.w - h.w));
}
// (re, im) -> (-im, re) for the two complex numbers of a float4: i times the value
__device__ __forceinline__ float4 rot4(float4 a) { return make_float4(-a.y, a.x, -a.w, a.z); }

// DRAIN: the accumulator is double-buffered in tensor memory (columns [0,128) and [128,256), Re
// then Im, N <= 64) and emptied every kDrain chunks into FP32 registers of the epilogue warps
// (round-to-nearest adds).  The tensor core's own accumulation truncates; draining keeps each
// truncated chain to 6 kDrain MMAs, so the result keeps FP32 accuracy over long contractions.
constexpr int kDrain = 2;

template <bool CONJ, int kStages, bool DRAIN>
__global__ void __launch_bounds__(kThreads, 1)
    k_tc_cgemm(const __grid_constant__ CUtensorMap amap, const __grid_constant__ CUtensorMap bmap,
               const TcJob* __restrict__ jobs, const TcArgs args, int* __restrict__ status) {
  extern __shared__ unsigned char dsm_raw[];
  unsigned char* sm = reinterpret_cast<unsigned char*>((reinterpret_cast<uintptr_t>(dsm_raw) + 1023) & ~uintptr_t(1023));
  __shared__ __align__(8) uint64_t bar_full[kStages], bar_ready[kStages], bar_empty[kStages], bar_acc[2], bar_drained[2];
  __shared__ uint32_t tmem_holder;
  __shared__ volatile int abort_flag;

  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const TcJob job = jobs[blockIdx.x / args.mtiles];
  const int mt = blockIdx.x % args.mtiles;
  const int m_valid = min(128, job.m_rows - mt * 128);
  if (m_valid <= 0) return;  // uniform over the CTA, before any shared state is touched
  const int a_y = job.a_y + mt * 128;
  const int nk = job.nslab * job.nchunk;
  const int abox = args.a_box;
  const int gcount = job.g_count, grows = gcount > 1 ? job.g_rows : m_valid;
  const int a_boxes_g = (grows + abox - 1) / abox;         // A boxes per row group
  const int a_rows = gcount > 1 ? gcount * grows : a_boxes_g * abox;  // tile rows that are loaded
  const int b_boxes = (job.n_valid + 31) >> 5;
  const uint32_t tx_bytes =
      (uint32_t)(gcount * a_boxes_g * abox * 64) + (uint32_t)(b_boxes * (CONJ ? 1 : 4)) * 2048u;
  const int n_int = DRAIN ? (nk + kDrain - 1) / kDrain : 1;  // accumulation intervals
  constexpr uint32_t kImOff = DRAIN ? 64u : 128u;            // Im accumulator column offset

  if (threadIdx.x == 0) {
    abort_flag = 0;
    for (int s = 0; s < kStages; ++s) {
      mbar_init(su32(&bar_full[s]), 1);
      mbar_init(su32(&bar_ready[s]), 128);
      mbar_init(su32(&bar_empty[s]), 1);
    }
    for (int b = 0; b < 2; ++b) {
      mbar_init(su32(&bar_acc[b]), 1);
      mbar_init(su32(&bar_drained[b]), 128);
    }
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
  }
  if (warp == 1) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(su32(&tmem_holder)),
                 "r"(kTmemCols)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  tc_before();
  __syncthreads();
  tc_after();
  const uint32_t tmem = tmem_holder;

  if (warp == 0) {
    if (lane == 0) {
      // ---- producer: TMA boxes of one chunk per stage
      int issued_round[kStages];
      for (int s = 0; s < kStages; ++s) issued_round[s] = -1;
      for (int kk = 0; kk < nk; ++kk) {
        const int s = kk % kStages, round = kk / kStages;
        if (round > 0 && !mbar_wait(su32(&bar_empty[s]), (round - 1) & 1, &abort_flag)) break;
        const int slab = kk / job.nchunk, ch = kk - slab * job.nchunk;
        const int ax = job.a_x + 16 * ch, bx = job.b_x + 16 * ch;
        const int az = job.a_z + slab * job.a_dz, bz = job.b_z + slab * job.b_dz;
        const uint32_t full = su32(&bar_full[s]);
        const uint32_t st = su32(sm + s * kStageBytes);
        mbar_expect_tx(full, tx_bytes);
        for (int g = 0; g < gcount; ++g)
          for (int i = 0; i < a_boxes_g; ++i)
            tma_load3(st + (g * grows + i * abox) * 64, &amap, ax, a_y + abox * i, az + g * job.g_dz, full);
        if (CONJ) {
          for (int i = 0; i < b_boxes; ++i)
            tma_load3(st + 2 * kTileBytes + i * 2048, &bmap, bx, job.b_y + 32 * i, bz, full);
        } else {
          for (int v = 0; v < 4; ++v)
            for (int i = 0; i < b_boxes; ++i)
              tma_load3(st + (2 + v) * kTileBytes + i * 2048, &bmap, bx, job.b_y + 32 * i, 4 * bz + v, full);
        }
        issued_round[s] = round;
      }
      // copies still in flight must land before the CTA exits
      for (int s = 0; s < kStages; ++s)
        if (issued_round[s] >= 0) mbar_wait(su32(&bar_full[s]), issued_round[s] & 1, &abort_flag, false);
    }
  } else if (warp == 1) {
    if (lane == 0) {
      // ---- MMA issuer: 2 K-steps of 8 per chunk, three TF32 products per real contraction
      const uint32_t idesc = tf32_idesc(job.n_mma);
      uint32_t t_re = tmem, t_im = tmem + kImOff;
      bool fresh = true;  // next MMA into each accumulator overwrites it
      int committed = -1;  // last interval whose completion was committed
      for (int kk = 0; kk < nk; ++kk) {
        if (DRAIN && kk % kDrain == 0) {
          const int i = kk / kDrain, b = i & 1;
          if (i >= 2 && !mbar_wait(su32(&bar_drained[b]), ((i - 2) >> 1) & 1, &abort_flag)) break;
          t_re = tmem + 128u * b;
          t_im = t_re + kImOff;
          fresh = true;
        }
        const int s = kk % kStages, round = kk / kStages;
        if (!mbar_wait(su32(&bar_ready[s]), round & 1, &abort_flag)) break;
        tc_after();
        const uint32_t base = su32(sm + s * kStageBytes);
#pragma unroll
        for (int sub = 0; sub < 2; ++sub) {
          const uint32_t o = 32u * sub;
          const uint64_t ah = sw64_desc(base + o), al = sw64_desc(base + kTileBytes + o);
          const uint64_t b1h = sw64_desc(base + 2 * kTileBytes + o), b1l = sw64_desc(base + 3 * kTileBytes + o);
          const uint64_t b2h = sw64_desc(base + 4 * kTileBytes + o), b2l = sw64_desc(base + 5 * kTileBytes + o);
          const uint32_t acc = (fresh && sub == 0) ? 0u : 1u;
          umma_tf32(t_re, al, b1h, idesc, acc);
          umma_tf32(t_re, ah, b1l, idesc, 1u);
          umma_tf32(t_re, ah, b1h, idesc, 1u);
          umma_tf32(t_im, al, b2h, idesc, acc);
          umma_tf32(t_im, ah, b2l, idesc, 1u);
          umma_tf32(t_im, ah, b2h, idesc, 1u);
        }
        fresh = false;
        umma_commit(su32(&bar_empty[s]));
        if (DRAIN && (kk % kDrain == kDrain - 1 || kk == nk - 1)) {
          umma_commit(su32(&bar_acc[(kk / kDrain) & 1]));
          committed = kk / kDrain;
        }
      }
      // also after an abort: the remaining completion barriers track the MMAs in flight
      if (DRAIN) {
        for (int i = committed + 1; i < n_int; ++i) umma_commit(su32(&bar_acc[i & 1]));
      } else {
        umma_commit(su32(&bar_acc[0]));
      }
    }
  } else {
    // ---- splitter (head and tail of the staged operands), drains, epilogue
    const int t = threadIdx.x - 64;
    const int q = warp & 3;
    const int row = 32 * q + lane;
    const uint32_t lane_addr = tmem + ((uint32_t)(32 * q) << 16);
    float acc_re[DRAIN ? 64 : 1], acc_im[DRAIN ? 64 : 1];
#pragma unroll
    for (int j = 0; j < (DRAIN ? 64 : 1); ++j) acc_re[j] = acc_im[j] = 0.f;
    int next_drain = 0;
    bool drain_ok = true;
    auto drain = [&](int i) {
      const int b = i & 1;
      if (!mbar_wait(su32(&bar_acc[b]), (i >> 1) & 1, &abort_flag, false)) drain_ok = false;
      tc_after();
      const uint32_t base = lane_addr + 128u * b;
#pragma unroll
      for (int n0 = 0; n0 < 64; n0 += 16) {
        if (n0 < job.n_mma) {
          uint32_t re[16], im[16];
          tmem_ld16(base + n0, re);
          tmem_ld16(base + kImOff + n0, im);
          tmem_wait_ld();
#pragma unroll
          for (int j = 0; j < 16; ++j) {
            acc_re[(n0 + j) & (DRAIN ? 63 : 0)] += __uint_as_float(re[j]);
            acc_im[(n0 + j) & (DRAIN ? 63 : 0)] += __uint_as_float(im[j]);
          }
        }
      }
      tc_before();
      mbar_arrive(su32(&bar_drained[b]));
    };
    for (int kk = 0; kk < nk; ++kk) {
      const int s = kk % kStages, round = kk / kStages;
      if (!mbar_wait(su32(&bar_full[s]), round & 1, &abort_flag)) break;
      unsigned char* st = sm + s * kStageBytes;
      float4* ah = reinterpret_cast<float4*>(st);
      float4* al = reinterpret_cast<float4*>(st + kTileBytes);
      for (int i = t; i < a_rows * 4; i += 128) {
        const float4 x = ah[i], h = head4(x);
        ah[i] = h;
        al[i] = tail4(x, h);
      }
      if (CONJ) {
        float4* b1h = reinterpret_cast<float4*>(st + 2 * kTileBytes);
        float4* b1l = reinterpret_cast<float4*>(st + 3 * kTileBytes);
        float4* b2h = reinterpret_cast<float4*>(st + 4 * kTileBytes);
        float4* b2l = reinterpret_cast<float4*>(st + 5 * kTileBytes);
        for (int i = t; i < b_boxes * 128; i += 128) {
          const float4 x = b1h[i], h = head4(x), l = tail4(x, h);
          b1h[i] = h;
          b1l[i] = l;
          b2h[i] = rot4(h);
          b2l[i] = rot4(l);
        }
      }
      asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
      mbar_arrive(su32(&bar_ready[s]));
      // after the last chunk of interval i, empty the other buffer (interval i - 1)
      if (DRAIN && (kk % kDrain == kDrain - 1) && kk / kDrain >= 1) drain(next_drain++);
    }
    bool ok;
    if (DRAIN) {
      while (next_drain < n_int) drain(next_drain++);  // bounded waits; MMAs in flight finish first
      ok = drain_ok && !abort_flag;
    } else {
      // accumulators complete (bounded wait, regardless of an abort: MMAs in flight must finish)
      ok = mbar_wait(su32(&bar_acc[0]), 0, &abort_flag, false) && !abort_flag;
      tc_after();
    }
    const long long R = (long long)a_y + row;
    long long obase;
    long long ostride;
    if (args.mode == 0) {
      obase = job.out_off + row;
      ostride = 128;
    } else {
      obase = job.out_off + (R / args.Rs) * args.S1 + (R % args.Rs);
      ostride = args.S2;
    }
    const bool store = ok && (gcount > 1 ? (row < gcount * grows && row % grows < job.g_valid) : row < m_valid);
    auto put = [&](int n, float xr, float xi) {
      if (store && n < job.n_valid)
        args.out[obase + (long long)n * ostride] =
            make_float2(args.alpha.x * xr - args.alpha.y * xi, args.alpha.x * xi + args.alpha.y * xr);
    };
    if (DRAIN) {
#pragma unroll
      for (int j = 0; j < 64; ++j) put(j, acc_re[j & (DRAIN ? 63 : 0)], acc_im[j & (DRAIN ? 63 : 0)]);
    } else {
      for (int n0 = 0; n0 < job.n_mma; n0 += 16) {
        uint32_t re[16], im[16];
        tmem_ld16(lane_addr + n0, re);
        tmem_ld16(lane_addr + kImOff + n0, im);
        tmem_wait_ld();
#pragma unroll
        for (int j = 0; j < 16; ++j) put(n0 + j, __uint_as_float(re[j]), __uint_as_float(im[j]));
      }
    }
  }
  tc_before();
  __syncthreads();
  if (warp == 1) {
    __syncwarp();
    tc_after();
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(kTmemCols) : "memory");
  }
  if (threadIdx.x == 0 && abort_flag) atomicExch(status, (int)DEV_TIMEOUT);
}

// out[tile] = alpha * sum over the tile's units of their FP32 partial tiles ([n][128] slots),
// summed in FP64 in a fixed order.
__global__ void k_tc_reduce(const TcTile* __restrict__ tiles, const float2* __restrict__ partial,
                            double2* __restrict__ out, double2 alpha, long long slot) {
  const TcTile T = tiles[blockIdx.x];
  const int n = T.m_valid * T.n_valid;
  for (int e = threadIdx.x; e < n; e += blockDim.x) {
    const int j = e / T.m_valid, m = e - j * T.m_valid;  // consecutive threads read consecutive rows
    const float2* p = partial + (long long)T.unit_begin * slot + (long long)(T.pn0 + j) * 128 + T.pm0 + m;
    double sx = 0.0, sy = 0.0;
    for (int u = 0; u < T.unit_count; ++u) {
      const float2 v = p[(long long)u * T.unit_stride * slot];
      sx += v.x;
      sy += v.y;
    }
    out[T.out_off + (long long)m * T.ld + j] = make_double2(alpha.x * sx - alpha.y * sy, alpha.x * sy + alpha.y * sx);
  }
}

// TF32 head and TF32 tail of a double: head + tail = x to about 2^-22 relative.
__device__ __forceinline__ void split_d(double x, float& h, float& l) {
  h = tf32_rn((float)x);
  l = tf32_rn((float)(x - (double)h));
}

// Dense B operands of the orbital right-multiplies from the packed G(tau) blocks.  For family 0
// B[n][k] = G[k][n] (the multiply D = X G), for family 1 B[n][k] = G[n][k] (D = X G^T).  Layout
// [fam][t][w][variant][n][2 nao] floats, variants (conj B) head, tail, (i conj B) head, tail.
__global__ void k_tc_g_operands(const double2* __restrict__ G, long long g_elems, const long long* __restrict__ g_off,
                                const int* __restrict__ bstart, const int* __restrict__ bsize,
                                const long long* __restrict__ bdoff, int nt, int nw, int nao, int fam0, int nfam,
                                float* __restrict__ out) {
  const long long per = (long long)nao * nao;
  const long long total = (long long)nfam * nt * nw * per;
  for (long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x; e < total;
       e += (long long)gridDim.x * blockDim.x) {
    const int k = (int)(e % nao);
    const int n = (int)((e / nao) % nao);
    const long long tw = e / per;  // (fam, t, w)
    const int w = (int)(tw % nw);
    const int t = (int)((tw / nw) % nt);
    const int fam = fam0 + (int)(tw / ((long long)nw * nt));
    const int r = fam == 0 ? k : n, cc = fam == 0 ? n : k;
    double2 g = make_double2(0.0, 0.0);
    const int* st = bstart + (long long)w * nao;
    if (st[r] == st[cc]) {
      const int b0 = st[r], bn = bsize[(long long)w * nao + r];
      g = G[(long long)t * g_elems + g_off[w] + bdoff[(long long)w * nao + r] + (long long)(r - b0) * bn + (cc - b0)];
    }
    // conj(B) = (re, -im); i conj(B) = (im, re)
    float h, l;
    float* base = out + (tw * 4) * per * 2 + (long long)n * 2 * nao + 2 * k;
    const long long vs = per * 2;
    split_d(g.x, h, l); base[0] = h; base[vs] = l;  base[2 * vs + 1] = h; base[3 * vs + 1] = l;
    split_d(-g.y, h, l); base[1] = h; base[vs + 1] = l;
    split_d(g.y, h, l); base[2 * vs] = h; base[3 * vs] = l;
  }
}

// B operands of the auxiliary multiply X2 = P^T X1 per block: B[n][d + 2 (A - s) + c] = comp_c(P[A][s + n]),
// d = (2 s) mod 4 so that the A operand's window starts on a 16-byte boundary.  Layout
// [tl][inst][variant][pt_rows][pt_k] floats for tau values t0 .. t0 + ntl - 1.
__global__ void k_tc_p_operands(const double2* __restrict__ P, long long p_elems, int t0, int ntl,
                                const int* __restrict__ info, const long long* __restrict__ boff, int ninst, int rows,
                                int kp, float* __restrict__ out) {
  const long long per = (long long)rows * kp;
  const long long total = (long long)ntl * ninst * per;
  for (long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x; e < total;
       e += (long long)gridDim.x * blockDim.x) {
    const int x = (int)(e % kp);
    const int n = (int)((e / kp) % rows);
    const long long ti = e / per;
    const int inst = (int)(ti % ninst);
    const int tl = (int)(ti / ninst);
    const int nb = info[3 * inst + 1], d = info[3 * inst + 2];
    const int kk = x - d;
    float v[4] = {0.f, 0.f, 0.f, 0.f};
    if (n < nb && kk >= 0 && kk < 2 * nb) {
      const int A = kk >> 1, comp = kk & 1;
      const double2 p = P[(long long)(t0 + tl) * p_elems + boff[inst] + (long long)A * nb + n];
      // conj(B) = (re, -im); i conj(B) = (im, re)
      const double c1 = comp == 0 ? p.x : -p.y, c2 = comp == 0 ? p.y : p.x;
      split_d(c1, v[0], v[1]);
      split_d(c2, v[2], v[3]);
    }
    float* base = out + (ti * 4) * per + (long long)n * kp + x;
    base[0] = v[0];
    base[per] = v[1];
    base[2 * per] = v[2];
    base[3 * per] = v[3];
  }
}

// Vt[p][i][A][a] = (complex64) V[p][A][i][a]
__global__ void k_tc_v_transpose(const double2* __restrict__ V, float2* __restrict__ Vt, long long npairs, int naux,
                                 int nao) {
  const long long vs = (long long)naux * nao * nao;
  const long long total = npairs * vs;
  for (long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x; e < total;
       e += (long long)gridDim.x * blockDim.x) {
    const int a = (int)(e % nao);
    const int A = (int)((e / nao) % naux);
    const int i = (int)((e / ((long long)nao * naux)) % nao);
    const long long p = e / vs;
    const double2 v = V[p * vs + ((long long)A * nao + i) * nao + a];
    Vt[e] = make_float2((float)v.x, (float)v.y);
  }
}

inline unsigned gridn(long long work, int threads) {
  long long b = (work + threads - 1) / threads;
  return (unsigned)std::max<long long>(1, std::min<long long>(b, 152LL * 64));
}

PFN_cuTensorMapEncodeTiled_v12000 g_encode = nullptr;
std::mutex g_encode_mu;

sgw_status get_encode(sgw_ctx* c) {
  std::lock_guard<std::mutex> lock(g_encode_mu);
  if (g_encode) return SGW_OK;
  void* fn = nullptr;
  cudaDriverEntryPointQueryResult q;
  cudaError_t e = cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &fn, 12000, cudaEnableDefault, &q);
  if (e != cudaSuccess || q != cudaDriverEntryPointSuccess || !fn)
    return c->fail(SGW_ERR_CUDA, "cuTensorMapEncodeTiled is not available from the driver");
  g_encode = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(fn);
  return SGW_OK;
}

// 3-D map of FP32 data: dims (kreals, rows, slabs), boxes of 16 reals x box_rows rows, 64-byte swizzle,
// zero fill outside the tensor.
sgw_status make_map(sgw_ctx* c, CUtensorMap* m, const void* base, long long kreals, long long rows, long long slabs,
                    long long row_bytes, long long slab_bytes, int box_rows = 32) {
  CKS(get_encode(c));
  if ((reinterpret_cast<uintptr_t>(base) & 15) || (row_bytes & 15) || (slab_bytes & 15) || (kreals & 3))
    return c->fail(SGW_ERR_ARG, "tensor-core operand not 16-byte aligned");
  cuuint64_t dims[3] = {(cuuint64_t)kreals, (cuuint64_t)rows, (cuuint64_t)slabs};
  cuuint64_t strides[2] = {(cuuint64_t)row_bytes, (cuuint64_t)slab_bytes};
  cuuint32_t box[3] = {16, (cuuint32_t)box_rows, 1};
  cuuint32_t es[3] = {1, 1, 1};
  CUresult r = g_encode(m, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 3, const_cast<void*>(base), dims, strides, box, es,
                        CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_64B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                        CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  if (r != CUDA_SUCCESS) return c->fail(SGW_ERR_CUDA, "cuTensorMapEncodeTiled failed (" + std::to_string((int)r) + ")");
  return SGW_OK;
}

constexpr int kMaxDev = 64;
bool g_attr_done[2][2][2][kMaxDev] = {};

// Short contractions (the orbital right-multiplies, a few chunks each) use two stages, so that two
// CTAs share an SM and one's epilogue overlaps the other's loads; long ones use four.
template <bool CONJ, int STAGES, bool DRAIN>
sgw_status launch_gemm(sgw_ctx* c, const CUtensorMap& am, const CUtensorMap& bm, const TcJob* jobs, long long njobs,
                       const TcArgs& a, cudaStream_t st) {
  if (njobs <= 0) return SGW_OK;
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDev) return c->fail(SGW_ERR_CUDA, "no current device");
  bool& done = g_attr_done[CONJ][STAGES == 4][DRAIN][dev];
  if (!done) {
    cudaError_t e = cudaFuncSetAttribute(k_tc_cgemm<CONJ, STAGES, DRAIN>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         smem_bytes(STAGES));
    if (e != cudaSuccess) return c->fail(SGW_ERR_CUDA, std::string("tensor-core kernel attribute: ") + cudaGetErrorString(e));
    done = true;
  }
  const long long grid = njobs * a.mtiles;
  if (grid > 0x7fffffffLL) return c->fail(SGW_ERR_ARG, "tensor-core launch too large");
  k_tc_cgemm<CONJ, STAGES, DRAIN><<<(unsigned)grid, kThreads, smem_bytes(STAGES), st>>>(am, bm, jobs, a, c->d_status);
  return SGW_OK;
}

template <typename T>
sgw_status up(sgw_ctx* c, T*& d, const std::vector<T>& h) {
  if (d) cudaFree(d);
  d = nullptr;
  if (h.empty()) return SGW_OK;
  if (cudaMalloc(&d, h.size() * sizeof(T)) != cudaSuccess) return c->fail(SGW_ERR_OOM, "tensor-core tables");
  if (cudaMemcpy(d, h.data(), h.size() * sizeof(T), cudaMemcpyHostToDevice) != cudaSuccess)
    return c->fail(SGW_ERR_CUDA, "uploading tensor-core tables");
  return SGW_OK;
}
template <typename T>
void fr(T*& p) {
  if (p) cudaFree(p);
  p = nullptr;
}

int round16(int n) { return (n + 15) & ~15; }
long long al256(long long bytes) { return (bytes + 255) & ~255LL; }

// Contraction chunks per split-K unit (a unit's FP32 partial tile is added to the others in FP64).
long long kchunk_target(bool drained) {
  const char* s = std::getenv(drained ? "SGW_TC_KCHUNK" : "SGW_TC_KCHUNK_UNDRAINED");
  long long v = s ? std::atoll(s) : (drained ? 128 : 16);
  return std::max(1LL, v);
}

struct KRange {
  int slab0, nslab, c0, nch;
};
// Split a contraction of nslab slabs x nchunk chunks into units of about `target` chunks.
std::vector<KRange> split_k(int nslab, int nchunk, long long target) {
  std::vector<KRange> out;
  if (nchunk >= target) {
    const int pieces = (int)((nchunk + target - 1) / target);
    const int per = (nchunk + pieces - 1) / pieces;
    for (int s = 0; s < nslab; ++s)
      for (int c0 = 0; c0 < nchunk; c0 += per) out.push_back({s, 1, c0, std::min(per, nchunk - c0)});
  } else {
    const int spu = (int)std::max<long long>(1, target / nchunk);
    for (int s0 = 0; s0 < nslab; s0 += spu) out.push_back({s0, std::min(spu, nslab - s0), 0, nchunk});
  }
  return out;
}

// Units of one Gram output block (rows [r0, r0 + nb) of A against rows [c0, c0 + nb) of B, or the
// given extents), tiles of 128 x ntile, ordered K range first so that the tiles of one K range run
// side by side and share their operand loads in L2.  Appends jobs and reduction tiles.
void gram_block(std::vector<TcJob>& jobs, std::vector<TcTile>& tiles, long long slot0, long long slot,
                const TcJob& proto, int mrows, int ncols, int ntile, int nslab, int nchunk, bool drained,
                long long out_base, int ld) {
  const int mts = (mrows + 127) / 128, nts = (ncols + ntile - 1) / ntile;
  const std::vector<KRange> kr = split_k(nslab, nchunk, kchunk_target(drained));
  const long long first = (long long)jobs.size() - slot0;
  for (const KRange& r : kr)
    for (int mi = 0; mi < mts; ++mi)
      for (int ni = 0; ni < nts; ++ni) {
        TcJob j = proto;
        j.a_y += 128 * mi;
        j.b_y += ntile * ni;
        j.a_z += r.slab0 * proto.a_dz;
        j.b_z += r.slab0 * proto.b_dz;
        j.a_x += 16 * r.c0;
        j.b_x += 16 * r.c0;
        j.nslab = r.nslab;
        j.nchunk = r.nch;
        j.m_rows = std::min(128, mrows - 128 * mi);
        j.n_valid = std::min(ntile, ncols - ntile * ni);
        j.n_mma = round16(j.n_valid);
        j.out_off = ((long long)jobs.size() - slot0) * slot;
        jobs.push_back(j);
      }
  if (ld <= 0) return;  // caller adds its own reduction tiles
  for (int mi = 0; mi < mts; ++mi)
    for (int ni = 0; ni < nts; ++ni) {
      TcTile t{};
      t.out_off = out_base + (long long)(128 * mi) * ld + ntile * ni;
      t.ld = ld;
      t.m_valid = std::min(128, mrows - 128 * mi);
      t.n_valid = std::min(ntile, ncols - ntile * ni);
      t.pm0 = 0;
      t.pn0 = 0;
      t.unit_begin = (int)(first + mi * nts + ni);
      t.unit_count = (int)kr.size();
      t.unit_stride = mts * nts;
      tiles.push_back(t);
    }
}

// Units of one small Gram block for several tau values at once: group g of the 128-row tile holds
// the block's rows at tau tg + g (groups R = nb rounded to 8 rows apart, slabs a_zg apart), all
// against the same B rows.  Appends the jobs and one reduction tile per tau value.
// Returns (first unit, unit count) so that callers can add further reduction tiles.
std::pair<long long, int> gram_stacked(std::vector<TcJob>& jobs, std::vector<TcTile>& tiles, long long slot0,
                                       long long slot, const TcJob& proto, int nb, int G, int a_zg, int nslab,
                                       int nchunk, const long long* out_base, int ld, int pm0, int pn0, int m_out,
                                       int n_out) {
  const int R = (nb + 7) & ~7;
  const std::vector<KRange> kr = split_k(nslab, nchunk, kchunk_target(true));
  const long long first = (long long)jobs.size() - slot0;
  for (const KRange& r : kr) {
    TcJob j = proto;
    j.a_z += r.slab0 * proto.a_dz;
    j.b_z += r.slab0 * proto.b_dz;
    j.a_x += 16 * r.c0;
    j.b_x += 16 * r.c0;
    j.nslab = r.nslab;
    j.nchunk = r.nch;
    j.g_count = G;
    j.g_rows = R;
    j.g_valid = nb;
    j.g_dz = a_zg;
    j.m_rows = G * R;
    j.n_valid = nb;
    j.n_mma = round16(nb);
    j.out_off = ((long long)jobs.size() - slot0) * slot;
    jobs.push_back(j);
  }
  for (int g = 0; out_base && g < G; ++g) {
    TcTile t{};
    t.out_off = out_base[g];
    t.ld = ld;
    t.m_valid = m_out;
    t.n_valid = n_out;
    t.pm0 = g * R + pm0;
    t.pn0 = pn0;
    t.unit_begin = (int)first;
    t.unit_count = (int)kr.size();
    t.unit_stride = 1;
    tiles.push_back(t);
  }
  return {first, (int)kr.size()};
}

int qindex(const sgw_ctx* c, int k1, int k2) {
  const int n1 = c->p.nk[0], n2 = c->p.nk[1], n3 = c->p.nk[2];
  auto iv = [&](int k, int d) { return d == 0 ? k / (n2 * n3) : d == 1 ? (k / n3) % n2 : k % n3; };
  int a = iv(k1, 0) - iv(k2, 0), b = iv(k1, 1) - iv(k2, 1), cc = iv(k1, 2) - iv(k2, 2);
  a = ((a % n1) + n1) % n1; b = ((b % n2) + n2) % n2; cc = ((cc % n3) + n3) % n3;
  return (a * n2 + b) * n3 + cc;
}

long long tc_nc(const sgw_ctx* c) {
  const long long vs = (long long)c->naux * c->nao * c->nao, np = (long long)c->nwedge * c->Nk;
  const char* s = std::getenv("SGW_WORKSPACE_GB");
  const double gb = s ? std::atof(s) : 24.0;
  const double budget = gb * 1e9;
  long long nc = (long long)(budget * 0.6 / (2.0 * np * vs * sizeof(float2)));
  return std::max(1LL, std::min<long long>(nc, c->nt));
}

sgw_status tables_common(sgw_ctx* c, TcPlan& T) {
  if (T.d_ao_start) return SGW_OK;
  const int nw = c->nwedge, nao = c->nao;
  std::vector<int> bs((size_t)nw * nao), bz((size_t)nw * nao);
  std::vector<long long> bd((size_t)nw * nao), go(nw);
  for (int w = 0; w < nw; ++w) {
    const Partition& P = c->part_ao[w];
    for (int v = 0; v < nao; ++v) {
      bs[(size_t)w * nao + v] = P.starts[v];
      bz[(size_t)w * nao + v] = P.isize[v];
      bd[(size_t)w * nao + v] = P.doff[v];
    }
    go[w] = c->g_off[w];
  }
  CKS(up(c, T.d_ao_start, bs));
  CKS(up(c, T.d_ao_size, bz));
  CKS(up(c, T.d_ao_doff, bd));
  CKS(up(c, T.d_g_off, go));
  return SGW_OK;
}

}  // namespace

namespace sgw {

bool tc_supported(const sgw_ctx* c) {
  const char* s = std::getenv("SGW_TC");
  if (s && std::strcmp(s, "0") == 0) return false;
  return c->p.precision == SGW_MIXED_FP32 && c->nao % 2 == 0 && c->naux % 2 == 0 && c->nao <= 128;
}

void tc_free(sgw_ctx* c) {
  if (!c->tc) return;
  TcPlan& T = *c->tc;
  fr(T.d_vg); fr(T.d_gvg); fr(T.d_pg); fr(T.d_svg); fr(T.d_pvg); fr(T.d_sg); fr(T.d_pr); fr(T.d_sr);
  fr(T.d_ao_start); fr(T.d_ao_size); fr(T.d_ao_doff); fr(T.d_g_off); fr(T.d_ab_info); fr(T.d_ab_off);
  delete c->tc;
  c->tc = nullptr;
}

// Interaction tensor for the tensor-core chains: orientation 0 keeps [pair][Q][i][j] (complex64),
// orientation 1 is stored as [pair][i][A][a] so that the self-energy contractions read it K-major.
void tc_store_v(const sgw_ctx* c, int which, const double2* V, float2* out, long long npairs, cudaStream_t st) {
  const long long n = npairs * (long long)c->naux * c->nao * c->nao;
  if (n <= 0) return;
  if (which == 0) {
    to_c64(V, out, n, st);
  } else {
    k_tc_v_transpose<<<gridn(n, 256), 256, 0, st>>>(V, out, npairs, c->naux, c->nao);
  }
}

static sgw_status build_p0(sgw_ctx* c) {
  TcPlan& T = *c->tc;
  if (T.built_p0) return SGW_OK;
  CKS(tables_common(c, T));
  const int Nk = c->Nk, nw = c->nwedge, nt = c->nt, nao = c->nao, naux = c->naux;
  const long long np = (long long)nw * Nk;
  const int nc = (int)tc_nc(c);
  T.nc_p0 = nc;
  const int rows = naux * nao;
  T.mt_vg = (rows + 127) / 128;
  std::vector<TcJob> vg, gvg, pg;
  std::vector<TcTile> pr;
  T.vg_start.assign(nt + 1, 0); T.gvg_start.assign(nt + 1, 0); T.pg_start.assign(nt + 1, 0); T.pr_start.assign(nt + 1, 0);
  const int kq = 2 * nao * nao;
  const int nch_g = (kq + 15) / 16, nch_o = (2 * nao + 15) / 16;
  for (int t = 0; t < nt; ++t) {
    const int tl = t % nc;
    T.vg_start[t] = vg.size(); T.gvg_start[t] = gvg.size();
    for (long long p = 0; p < np; ++p) {
      const int k1 = c->pair_k1[0][p], k2 = c->pair_k2[0][p];
      TcJob j{};
      j.a_y = 0; j.a_z = (int)p; j.b_y = 0;
      j.b_z = (int)(((long long)0 * nt + t) * nw + c->rep[k2]);
      j.a_x = 0; j.b_x = 0; j.nslab = 1; j.nchunk = nch_o; j.a_dz = 0; j.b_dz = 0;
      j.m_rows = rows; j.n_valid = nao; j.n_mma = round16(nao);
      j.out_off = ((long long)tl * np + p) * rows * nao;
      vg.push_back(j);
      TcJob g = j;
      g.a_z = (int)((long long)tl * np + p);
      g.b_z = (int)(((long long)1 * nt + (nt - 1 - t)) * nw + c->rep[k1]);
      gvg.push_back(g);
    }
  }
  // Gram units per tau chunk: blocks up to 64 stack several tau values in one tile
  for (int t0 = 0; t0 < nt; t0 += nc) {
    const int t1 = std::min(nt, t0 + nc);
    const long long slot0 = (long long)pg.size();
    for (int t = t0; t < t1; ++t) { T.pg_start[t] = pg.size(); T.pr_start[t] = pr.size(); }
    for (size_t b = 0; b < c->auxb_off.size(); ++b) {
      const int w = c->auxb_w[b], nb = c->auxb_n[b], s = c->auxb_start[b];
      TcJob j{};
      j.a_y = s; j.a_dz = 1;
      j.b_y = s; j.b_z = (int)((long long)w * Nk); j.b_dz = 1;
      if (nb <= 64) {
        const int G = 128 / ((nb + 7) & ~7);
        for (int tg = t0; tg < t1; tg += G) {
          const int Gp = std::min(G, t1 - tg);
          j.a_z = (int)((long long)(tg - t0) * np + (long long)w * Nk);
          std::vector<long long> ob(Gp);
          for (int g = 0; g < Gp; ++g) ob[g] = (long long)(tg + g) * c->p_elems + c->auxb_off[b];
          gram_stacked(pg, pr, slot0, kSlotD, j, nb, Gp, (int)np, Nk, nch_g, ob.data(), nb, 0, 0, nb, nb);
        }
      } else {
        for (int t = t0; t < t1; ++t) {
          j.a_z = (int)((long long)(t - t0) * np + (long long)w * Nk);
          gram_block(pg, pr, slot0, kSlotD, j, nb, nb, 64, Nk, nch_g, true,
                     (long long)t * c->p_elems + c->auxb_off[b], nb);
        }
      }
    }
  }
  T.vg_start[nt] = vg.size(); T.gvg_start[nt] = gvg.size(); T.pg_start[nt] = pg.size(); T.pr_start[nt] = pr.size();
  T.max_units_p0 = 0;
  for (int t0 = 0; t0 < nt; t0 += nc) {
    const int t1 = std::min(nt, t0 + nc);
    T.max_units_p0 = std::max(T.max_units_p0, T.pg_start[t1] - T.pg_start[t0]);
  }
  T.fl_vg = T.fl_gvg = T.fl_pg = 0;
  for (long long p = 0; p < np; ++p) {
    T.fl_vg += 8.0 * naux * nao * (double)c->part_ao[c->rep[c->pair_k2[0][p]]].elems;
    T.fl_gvg += 8.0 * naux * nao * (double)c->part_ao[c->rep[c->pair_k1[0][p]]].elems;
  }
  for (int w = 0; w < nw; ++w) T.fl_pg += 8.0 * Nk * (double)nao * nao * c->part_aux[w].elems;
  CKS(up(c, T.d_vg, vg));
  CKS(up(c, T.d_gvg, gvg));
  CKS(up(c, T.d_pg, pg));
  CKS(up(c, T.d_pr, pr));
  T.built_p0 = true;
  return SGW_OK;
}

static sgw_status build_sigma(sgw_ctx* c) {
  TcPlan& T = *c->tc;
  if (T.built_sigma) return SGW_OK;
  CKS(tables_common(c, T));
  const int Nk = c->Nk, nw = c->nwedge, nt = c->nt, nao = c->nao, naux = c->naux;
  const long long np = (long long)nw * Nk;
  const int nc = (int)tc_nc(c);
  T.nc_s = nc;
  T.drain_s = nao <= 64;
  T.slot_s = T.drain_s ? kSlotD : kSlot;
  const long long vs = (long long)naux * nao * nao;
  // auxiliary block instances (all wedge q): start, size, delta; P^T operand extents
  const int ninst = (int)c->auxb_off.size();
  T.ninst = ninst;
  std::vector<int> info(3 * (size_t)ninst);
  std::vector<long long> boff(ninst);
  int rmax = 0, kmax = 0;
  std::vector<std::vector<int>> wblocks(nw);
  for (int b = 0; b < ninst; ++b) {
    const int s = c->auxb_start[b], nb = c->auxb_n[b], d = (2 * s) & 3;
    info[3 * b] = s; info[3 * b + 1] = nb; info[3 * b + 2] = d;
    boff[b] = c->auxb_off[b];
    rmax = std::max(rmax, nb);
    kmax = std::max(kmax, (d + 2 * nb + 15) / 16 * 16);
    wblocks[c->auxb_w[b]].push_back(b);
  }
  T.pt_rows = rmax;
  T.pt_k = kmax;
  CKS(up(c, T.d_ab_info, info));
  CKS(up(c, T.d_ab_off, boff));
  const int rows_v = nao * naux, rows_x = nao * nao;
  T.mt_svg = (rows_v + 127) / 128;
  T.mt_pvg = (rows_x + 127) / 128;
  std::vector<TcJob> svg, pvg, sg;
  std::vector<TcTile> sr;
  T.svg_start.assign(nt + 1, 0); T.pvg_start.assign(nt + 1, 0); T.sg_start.assign(nt + 1, 0); T.sr_start.assign(nt + 1, 0);
  const int nch_o = (2 * nao + 15) / 16, kg = 2 * naux * nao, nch_g = (kg + 15) / 16;
  for (int t = 0; t < nt; ++t) {
    const int tl = t % nc;
    T.svg_start[t] = svg.size(); T.pvg_start[t] = pvg.size();
    for (long long p = 0; p < np; ++p) {
      const int k1 = c->pair_k1[1][p], k2 = c->pair_k2[1][p];
      TcJob j{};
      j.a_y = 0; j.a_z = (int)p; j.b_y = 0;
      j.b_z = (int)((long long)t * nw + c->rep[k2]);
      j.nslab = 1; j.nchunk = nch_o;
      j.m_rows = rows_v; j.n_valid = nao; j.n_mma = round16(nao);
      j.out_off = ((long long)tl * np + p) * vs;
      svg.push_back(j);
      const int wq = c->rep[qindex(c, k1, k2)];
      for (int b : wblocks[wq]) {
        const int s = info[3 * b], nb = info[3 * b + 1], d = info[3 * b + 2];
        for (int n0 = 0; n0 < nb; n0 += 64) {
          TcJob v{};
          v.a_y = 0; v.a_z = (int)((long long)tl * np + p);
          v.a_x = 2 * s - d;
          v.b_y = n0; v.b_z = tl * ninst + b;
          v.b_x = 0;
          v.nslab = 1; v.nchunk = (d + 2 * nb + 15) / 16;
          v.m_rows = rows_x; v.n_valid = std::min(64, nb - n0); v.n_mma = round16(v.n_valid);
          v.out_off = ((long long)tl * np + p) * vs + (long long)(s + n0) * nao;
          pvg.push_back(v);
        }
      }
    }
  }
  // Gram units per tau chunk: the whole nao x nao matrix per wedge point (the reduction picks the
  // diagonal blocks); up to 64 orbitals, several tau values share one tile
  for (int t0 = 0; t0 < nt; t0 += nc) {
    const int t1 = std::min(nt, t0 + nc);
    const long long slot0 = (long long)sg.size();
    for (int t = t0; t < t1; ++t) { T.sg_start[t] = sg.size(); T.sr_start[t] = sr.size(); }
    for (int w = 0; w < nw; ++w) {
      TcJob j{};
      j.a_y = 0; j.a_dz = 1;
      j.b_y = 0; j.b_z = (int)((long long)w * Nk); j.b_dz = 1;
      const int R = (nao + 7) & ~7;
      const int G = T.drain_s ? 128 / R : 1;
      for (int tg = t0; tg < t1; tg += G) {
        const int Gp = std::min(G, t1 - tg);
        j.a_z = (int)((long long)(tg - t0) * np + (long long)w * Nk);
        long long u0;
        int nunits;
        if (T.drain_s) {
          std::tie(u0, nunits) = gram_stacked(sg, sr, slot0, T.slot_s, j, nao, Gp, (int)np, Nk, nch_g, nullptr, 0, 0,
                                              0, 0, 0);
        } else {
          u0 = (long long)sg.size() - slot0;
          gram_block(sg, sr, slot0, T.slot_s, j, nao, nao, 128, Nk, nch_g, false, 0, 0);
          nunits = (int)((long long)sg.size() - slot0 - u0);
        }
        for (int g = 0; g < Gp; ++g)
          for (size_t b = 0; b < c->aob_off.size(); ++b) {
            if (c->aob_w[b] != w) continue;
            TcTile tile{};
            const int nb = c->aob_n[b], s = c->aob_start[b];
            tile.out_off = (long long)(tg + g) * c->g_elems + c->aob_off[b];
            tile.ld = nb; tile.m_valid = nb; tile.n_valid = nb; tile.pm0 = g * R + s; tile.pn0 = s;
            tile.unit_begin = (int)u0; tile.unit_count = nunits; tile.unit_stride = 1;
            sr.push_back(tile);
          }
      }
    }
  }
  T.svg_start[nt] = svg.size(); T.pvg_start[nt] = pvg.size(); T.sg_start[nt] = sg.size(); T.sr_start[nt] = sr.size();
  T.max_units_s = 0;
  for (int t0 = 0; t0 < nt; t0 += nc) {
    const int t1 = std::min(nt, t0 + nc);
    T.max_units_s = std::max(T.max_units_s, T.sg_start[t1] - T.sg_start[t0]);
  }
  T.fl_svg = T.fl_pvg = T.fl_sg = 0;
  for (long long p = 0; p < np; ++p) {
    const int k1 = c->pair_k1[1][p], k2 = c->pair_k2[1][p];
    T.fl_svg += 8.0 * naux * nao * (double)c->part_ao[c->rep[k2]].elems;
    T.fl_pvg += 8.0 * nao * nao * (double)c->part_aux[c->rep[qindex(c, k1, k2)]].elems;
  }
  for (int w = 0; w < nw; ++w) T.fl_sg += 8.0 * Nk * (double)naux * nao * c->part_ao[w].elems;
  CKS(up(c, T.d_svg, svg));
  CKS(up(c, T.d_pvg, pvg));
  CKS(up(c, T.d_sg, sg));
  CKS(up(c, T.d_sr, sr));
  T.built_sigma = true;
  return SGW_OK;
}

static sgw_status ensure_plan(sgw_ctx* c) {
  if (!c->tc) c->tc = new TcPlan();
  return SGW_OK;
}

sgw_status tc_polarization(sgw_ctx* c, const double2* G, double2* out, cudaStream_t st) {
  CKS(ensure_plan(c));
  CKS(build_p0(c));
  TcPlan& T = *c->tc;
  const int nt = c->nt, nw = c->nwedge, nao = c->nao, naux = c->naux, Nk = c->Nk, nc = T.nc_p0;
  const long long np = (long long)nw * Nk, vs = (long long)naux * nao * nao;
  const long long inter = (long long)nc * np * vs;  // complex64 elements
  const long long gop = 2LL * nt * nw * 4 * nao * 2 * nao;  // floats
  const long long b_z = al256(inter * 8), b_x = al256(inter * 8), b_g = al256(gop * 4),
                  b_p = al256(T.max_units_p0 * kSlotD * 8);
  CKS(ensure_workspace(c, (size_t)(b_z + b_x + b_g + b_p)));
  unsigned char* ws = reinterpret_cast<unsigned char*>(c->d_ws);
  float2* Zp = reinterpret_cast<float2*>(ws);
  float2* X = reinterpret_cast<float2*>(ws + b_z);
  float* Gop = reinterpret_cast<float*>(ws + b_z + b_x);
  float2* part = reinterpret_cast<float2*>(ws + b_z + b_x + b_g);
  run(c, "tc_prep", 0.0, 1, st, [&] {
    k_tc_g_operands<<<gridn(2LL * nt * nw * nao * nao, 256), 256, 0, st>>>(
        G, c->g_elems, T.d_g_off, T.d_ao_start, T.d_ao_size, T.d_ao_doff, nt, nw, nao, 0, 2, Gop);
  });
  CUtensorMap mV, mZ, mG;
  const long long rows = (long long)naux * nao;
  CKS(make_map(c, &mV, c->d_V32[0], 2 * nao, rows, np, 8LL * nao, vs * 8));
  CKS(make_map(c, &mZ, Zp, 2 * nao, rows, (long long)nc * np, 8LL * nao, vs * 8));
  CKS(make_map(c, &mG, Gop, 2 * nao, nao, 2LL * nt * nw * 4, 8LL * nao, 8LL * nao * nao));
  // Gram operands: rows Q, contracted (i, j) re/im
  CUtensorMap mXg, mVg;
  CKS(make_map(c, &mXg, X, 2LL * nao * nao, naux, (long long)nc * np, 8LL * nao * nao, vs * 8, 8));
  CKS(make_map(c, &mVg, c->d_V32[0], 2LL * nao * nao, naux, np, 8LL * nao * nao, vs * 8));
  const double alpha = c->p.loop_sign * (double)c->p.spin_factor / c->Nk;
  for (int t0 = 0; t0 < nt; t0 += nc) {
    const int t1 = std::min(nt, t0 + nc), ntc = t1 - t0;
    TcArgs a{};
    a.a_box = 32;
    a.mtiles = T.mt_vg; a.mode = 1; a.Rs = nao; a.S1 = (long long)nao * nao; a.S2 = nao;
    a.alpha = make_float2(1.f, 0.f); a.out = Zp;
    // Z'[A][j][c] = sum_d V[A][c][d] G^{k+q}(tau)[d][j]
    sgw_status s1 = SGW_OK, s2 = SGW_OK, s3 = SGW_OK;
    run(c, "p0_vg_tc", T.fl_vg * ntc, 1, st, [&] {
      s1 = launch_gemm<false, 2, false>(c, mV, mG, T.d_vg + T.vg_start[t0], T.vg_start[t1] - T.vg_start[t0], a, st);
    });
    CKS(s1);
    // X[A][i][j] = sum_c G^k(-tau)[i][c] Z'[A][j][c],  G(-tau_j) = -G(tau_{n-1-j})
    a.alpha = make_float2(-1.f, 0.f); a.out = X;
    run(c, "p0_gvg_tc", T.fl_gvg * ntc, 1, st, [&] {
      s2 = launch_gemm<false, 2, false>(c, mZ, mG, T.d_gvg + T.gvg_start[t0], T.gvg_start[t1] - T.gvg_start[t0], a, st);
    });
    CKS(s2);
    // P0 block tiles: sum over k and (i, j) of X[Q][(i,j)] conj(V[Q'][(i,j)])
    TcArgs g{};
    g.a_box = 8;
    g.mtiles = 1; g.mode = 0; g.Rs = 1; g.alpha = make_float2(1.f, 0.f); g.out = part;
    run(c, "p0_gram_tc", T.fl_pg * ntc, 1, st, [&] {
      s3 = launch_gemm<true, 4, true>(c, mXg, mVg, T.d_pg + T.pg_start[t0], T.pg_start[t1] - T.pg_start[t0], g, st);
    });
    CKS(s3);
    const long long r0 = T.pr_start[t0], r1 = T.pr_start[t1];
    run(c, "gram_reduce", 0.0, 1, st, [&] {
      if (r1 > r0) k_tc_reduce<<<(unsigned)(r1 - r0), 256, 0, st>>>(T.d_pr + r0, part, out, make_double2(alpha, 0.0), kSlotD);
    });
  }
  return SGW_OK;
}

sgw_status tc_self_energy(sgw_ctx* c, const double2* G, const double2* P, double2* out, cudaStream_t st) {
  CKS(ensure_plan(c));
  CKS(build_sigma(c));
  TcPlan& T = *c->tc;
  const int nt = c->nt, nw = c->nwedge, nao = c->nao, naux = c->naux, Nk = c->Nk, nc = T.nc_s;
  const long long np = (long long)nw * Nk, vs = (long long)naux * nao * nao;
  const long long inter = (long long)nc * np * vs;
  const long long gop = 1LL * nt * nw * 4 * nao * 2 * nao;
  const long long pop = (long long)nc * T.ninst * 4 * T.pt_rows * T.pt_k;
  const long long b_1 = al256(inter * 8), b_2 = al256(inter * 8), b_g = al256(gop * 4), b_pp = al256(pop * 4),
                  b_p = al256(T.max_units_s * T.slot_s * 8);
  CKS(ensure_workspace(c, (size_t)(b_1 + b_2 + b_g + b_pp + b_p)));
  unsigned char* ws = reinterpret_cast<unsigned char*>(c->d_ws);
  float2* X1 = reinterpret_cast<float2*>(ws);
  float2* X2 = reinterpret_cast<float2*>(ws + b_1);
  float* Gop = reinterpret_cast<float*>(ws + b_1 + b_2);
  float* Pop = reinterpret_cast<float*>(ws + b_1 + b_2 + b_g);
  float2* part = reinterpret_cast<float2*>(ws + b_1 + b_2 + b_g + b_pp);
  run(c, "tc_prep", 0.0, 1, st, [&] {
    k_tc_g_operands<<<gridn(1LL * nt * nw * nao * nao, 256), 256, 0, st>>>(
        G, c->g_elems, T.d_g_off, T.d_ao_start, T.d_ao_size, T.d_ao_doff, nt, nw, nao, 0, 1, Gop);
  });
  CUtensorMap mVt, mG, mX1, mP, mX2g, mVtg;
  const long long rows_v = (long long)nao * naux;
  CKS(make_map(c, &mVt, c->d_V32[1], 2 * nao, rows_v, np, 8LL * nao, vs * 8));
  CKS(make_map(c, &mG, Gop, 2 * nao, nao, 1LL * nt * nw * 4, 8LL * nao, 8LL * nao * nao));
  CKS(make_map(c, &mX1, X1, 2LL * naux, (long long)nao * nao, (long long)nc * np, 8LL * naux, vs * 8));
  CKS(make_map(c, &mP, Pop, T.pt_k, T.pt_rows, (long long)nc * T.ninst * 4, 4LL * T.pt_k, 4LL * T.pt_k * T.pt_rows));
  CKS(make_map(c, &mX2g, X2, 2LL * naux * nao, nao, (long long)nc * np, 8LL * naux * nao, vs * 8, 8));
  CKS(make_map(c, &mVtg, c->d_V32[1], 2LL * naux * nao, nao, np, 8LL * naux * nao, vs * 8));
  for (int t0 = 0; t0 < nt; t0 += nc) {
    const int t1 = std::min(nt, t0 + nc), ntc = t1 - t0;
    run(c, "tc_prep", 0.0, 1, st, [&] {
      k_tc_p_operands<<<gridn((long long)ntc * T.ninst * T.pt_rows * T.pt_k, 256), 256, 0, st>>>(
          P, c->p_elems, t0, ntc, T.d_ab_info, T.d_ab_off, T.ninst, T.pt_rows, T.pt_k, Pop);
    });
    sgw_status s1 = SGW_OK, s2 = SGW_OK, s3 = SGW_OK;
    // X1T[i][b][A] = sum_a V[A][i][a] G^{k2}(tau)[a][b]
    TcArgs a{};
    a.a_box = 32;
    a.mtiles = T.mt_svg; a.mode = 1; a.Rs = naux; a.S1 = (long long)nao * naux; a.S2 = naux;
    a.alpha = make_float2(1.f, 0.f); a.out = X1;
    run(c, "sigma_vg_tc", T.fl_svg * ntc, 1, st, [&] {
      s1 = launch_gemm<false, 2, false>(c, mVt, mG, T.d_svg + T.svg_start[t0], T.svg_start[t1] - T.svg_start[t0], a, st);
    });
    CKS(s1);
    // X2[i][A'][b] = sum_A P^q(tau)[A][A'] X1T[i][b][A]
    TcArgs b{};
    b.a_box = 32;
    b.mtiles = T.mt_pvg; b.mode = 1; b.Rs = nao; b.S1 = (long long)naux * nao; b.S2 = nao;
    b.alpha = make_float2(1.f, 0.f); b.out = X2;
    run(c, "sigma_pvg_tc", T.fl_pvg * ntc, 1, st, [&] {
      s2 = launch_gemm<false, 4, true>(c, mX1, mP, T.d_pvg + T.pvg_start[t0], T.pvg_start[t1] - T.pvg_start[t0], b, st);
    });
    CKS(s2);
    // Sigma tiles: sum over k2 and (A', b) of X2[i][(A',b)] conj(Vt[i'][(A',b)])
    TcArgs g{};
    g.a_box = 8;
    g.mtiles = 1; g.mode = 0; g.Rs = 1; g.alpha = make_float2(1.f, 0.f); g.out = part;
    run(c, "sigma_gram_tc", T.fl_sg * ntc, 1, st, [&] {
      const TcJob* jb = T.d_sg + T.sg_start[t0];
      const long long nj = T.sg_start[t1] - T.sg_start[t0];
      s3 = T.drain_s ? launch_gemm<true, 4, true>(c, mX2g, mVtg, jb, nj, g, st)
                     : launch_gemm<true, 4, false>(c, mX2g, mVtg, jb, nj, g, st);
    });
    CKS(s3);
    const long long r0 = T.sr_start[t0], r1 = T.sr_start[t1];
    run(c, "gram_reduce", 0.0, 1, st, [&] {
      if (r1 > r0)
        k_tc_reduce<<<(unsigned)(r1 - r0), 256, 0, st>>>(T.d_sr + r0, part, out, make_double2(-1.0 / c->Nk, 0.0),
                                                          T.slot_s);
    });
  }
  return SGW_OK;
}

}  // namespace sgw
