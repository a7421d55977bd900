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
// The contraction kernel is persistent and warp-specialised (one CTA per SM walking its units:
// a TMA producer warp, an MMA warp, a head/tail splitter warpgroup and two epilogue warpgroups;
// see k_tc_persist).  Every wait is bounded in time; a CTA that runs out of time records SGW
// status "timeout", drains its copies in flight, frees its tensor memory and returns.
#include <cuda.h>
#include <cudaTypedefs.h>

#include <algorithm>
#include <cmath>
#include <cstdio>
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
  int nslab = 1, nchunk = 1;  // contraction loop: nslab slabs x nchunk chunks of 32 reals
  int a_dz = 0, b_dz = 0;  // slab increments
  int m_rows = 0;          // rows of A the job covers (tiles of 128)
  int n_valid = 0, n_mma = 16;  // stored columns; MMA width (multiple of 16, <= 128)
  int pad = 0;
  long long out_off = 0;   // partial slot (Gram) or output base (affine store)
};
static_assert(sizeof(TcJob) == 64, "TcJob layout");

// Output tile of a Gram reduction over the partial tiles of its units (FP64 sum in order): element
// (m, j) of the output block is row pm0 + m pm_stride, column pn0 + j of each unit's partial tile.
struct alignas(16) TcTile {
  long long out_off;
  int ld, m_valid, n_valid, pm0, pm_stride, pn0, unit_begin, unit_count, unit_stride;
};

struct TcArgs {
  int mtiles;          // 128-row tiles per job
  int a_box;           // rows per A box of the A tensor map (32 or 128)
  int b_rows;          // rows per B box; the B variants sit b_rows rows apart in shared memory
  int mode;            // 0: FP32 partial tile [n][m] at out_off; 1: affine store
  long long Rs, S1, S2;  // affine store: out[out_off + (R / Rs) S1 + (R % Rs) + n S2], R = tile row
  float2 alpha;
  float2* out;
  unsigned long long wait_ns;  // limit of each pipeline wait (SGW_ERR_TIMEOUT beyond it)
};

// Cached jobs of the tensor-core chains.
struct TcPlan {
  long long pb = 0, pe = 0;            // pair range [pb, pe) of the orientation's pair list
  int nt_eff = 0;                      // tau values the P0 chain contracts (the reflection gives the rest)
  bool built_p0 = false, built_sigma = false;
  long long unit_p0 = 0, unit_s = 0;   // split-K unit length of the Gram reductions (chunks)
  bool tuned_p0 = false, tuned_s = false;
  int nc_p0 = 0, nc_s = 0;
  int nc_req_p0 = 0, nc_req_s = 0;         // tau chunk asked for (0: the largest the workspace allows)
  bool tuned_nc_p0 = false, tuned_nc_s = false;
  std::vector<long long> vg_start, gvg_start, pg_start, pr_start;            // per tau: first job / unit / tile
  std::vector<long long> svg_start, pvg_start, sg_start, sr_start;
  TcJob *d_vg = nullptr, *d_gvg = nullptr, *d_pg = nullptr, *d_svg = nullptr, *d_pvg = nullptr, *d_sg = nullptr;
  TcTile *d_pr = nullptr, *d_sr = nullptr;
  std::vector<long long> prp_start, srp_start;  // per tau: first reduction piece
  int2 *d_prp = nullptr, *d_srp = nullptr;
  long long max_units_p0 = 0, max_units_s = 0;
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

// One chunk of the contraction is 32 reals (a 128-byte swizzle row of FP32): an A tile of 128 rows
// and the four 64-row B variants (B1 head, B2 head, B1 tail, B2 tail) per stage.
constexpr int kChunkReals = 32;
constexpr int kRowBytes = 4 * kChunkReals;           // 128
constexpr int kABytes = 128 * kRowBytes;             // 16 KB
constexpr int kBVarBytes = 64 * kRowBytes;           // 8 KB
constexpr int kStageBytes = kABytes + 4 * kBVarBytes;  // 48 KB
// Drain waits (copies in flight, MMAs issued) always allow 2 s: a CTA must not exit while a copy
// into its shared memory can still land.  The pipeline waits use the context's limit (TcArgs).
constexpr unsigned long long kDrainNs = 2000000000ULL;
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
// Wait for the phase of the given parity; false once limit_ns have passed since the first failed
// try (sets *abort; a limit of 0 gives up at the first failed try) or once *abort is set by another
// role (if honour_abort).
__device__ bool mbar_wait(uint32_t bar, uint32_t parity, volatile int* abort, unsigned long long limit_ns,
                          bool honour_abort = true) {
  if (mbar_try(bar, parity)) return true;
  const unsigned long long t0 = gtime();
  while (true) {
    if (mbar_try(bar, parity)) return true;
    if (honour_abort && *abort) return false;
    if (gtime() - t0 >= limit_ns) {
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
__device__ __forceinline__ void tma_load4(uint32_t dst, const CUtensorMap* map, int x, int y, int v, int z,
                                          uint32_t bar) {
  asm volatile(
      "cp.async.bulk.tensor.4d.shared::cluster.global.tile.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3, %4, "
      "%5}], [%6];" ::"r"(dst),
      "l"(reinterpret_cast<uint64_t>(map)), "r"(x), "r"(y), "r"(v), "r"(z), "r"(bar)
      : "memory");
}
__device__ __forceinline__ void tc_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void tc_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }
// Shared-memory matrix descriptor: K-major, 128-byte swizzle, 8-row groups 1024 bytes apart.  The
// K steps of a chunk start 32, 64 and 96 bytes into the rows: the swizzle phase (address bits 7-9)
// is that of the 1024-byte aligned tile, so the base offset field stays 0.
__device__ __forceinline__ uint64_t sw128_desc(uint32_t saddr) {
  return (uint64_t)((saddr & 0x3FFFFu) >> 4) | ((uint64_t)1 << 16) | ((uint64_t)(1024 >> 4) << 32) |
         ((uint64_t)1 << 46) | ((uint64_t)2 << 61);
}
// Instruction descriptor: kind::tf32, FP32 accumulator, both operands K-major, M = 128.
__device__ __forceinline__ uint32_t tf32_idesc(int n) {
  return (1u << 4) | (2u << 7) | (2u << 10) | ((uint32_t)(n >> 3) << 17) | ((uint32_t)(128 >> 4) << 24);
}
// A operand in tensor memory (128 lanes = rows, 8 columns = the K step), B in shared memory
__device__ __forceinline__ void umma_tf32_ta(uint32_t d, uint32_t a_tmem, uint64_t b, uint32_t idesc, uint32_t acc) {
  asm volatile(
      "{\n.reg .pred p;\nsetp.ne.b32 p, %4, 0;\ntcgen05.mma.cta_group::1.kind::tf32 [%0], [%1], %2, %3, p;\n}" ::"r"(d),
      "r"(a_tmem), "l"(b), "r"(idesc), "r"(acc)
      : "memory");
}
__device__ __forceinline__ void tmem_st16(uint32_t taddr, const float* v) {
  asm volatile(
      "tcgen05.st.sync.aligned.32x32b.x16.b32 [%0], {%1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, "
      "%15, %16};" ::"r"(taddr),
      "f"(v[0]), "f"(v[1]), "f"(v[2]), "f"(v[3]), "f"(v[4]), "f"(v[5]), "f"(v[6]), "f"(v[7]), "f"(v[8]), "f"(v[9]),
      "f"(v[10]), "f"(v[11]), "f"(v[12]), "f"(v[13]), "f"(v[14]), "f"(v[15])
      : "memory");
}
__device__ __forceinline__ void tmem_wait_st() { asm volatile("tcgen05.wait::st.sync.aligned;" ::: "memory"); }
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

// Persistent, warp-specialised contraction kernel.  One CTA per SM walks the units
// u = blockIdx.x, blockIdx.x + gridDim.x, ...; the shared-memory stage ring and the
// tensor-memory accumulator ring run on across units, so the loads of one tile overlap the
// MMAs and the stores of the previous ones.
//   warps 0, 2, 3 TMA producers (one lane each): producer p issues the boxes of the chunks
//                 g = p (mod 3) of the CTA's chunk sequence, each into stage g mod 4 once the
//                 stage is free (an SM takes in about one box per 700-1000 clocks per issuing warp,
//                 whatever the box size, so the copies of consecutive chunks come from different
//                 warps)
//   warp 1        tensor-memory owner; one lane issues 12 MMAs per chunk (4 K steps of 8 x 3)
//   warps 4-7     splitter: TF32 head and tail of the staged A rows into tensor memory (and the
//                 B variants of the Gram form in shared memory)
//   warps 8-15    epilogue, two warpgroups, each one half of the accumulator columns (a warp
//                 reads the 32 tensor-memory lanes of its rank within the warpgroup)
// Tensor memory: 2 accumulator buffers of 128 columns (Re 64, Im 64) in [0, 256), the A head and
// tail of the four stages (32 + 32 columns each) in [256, 512).  DRAIN: every kDrain chunks the
// MMA warp moves to the next buffer and the epilogue adds the finished one into round-to-nearest
// FP32 registers (the tensor core's own accumulation truncates), storing them at the end of the
// unit.  Without DRAIN: one buffer per unit, read once.
// All waits are bounded in time (status SGW_ERR_TIMEOUT, copies drained, tensor memory freed).
constexpr int kDrain = 1;
constexpr int kPThreads = 512;
constexpr int kPStages = 4;
constexpr int kNProd = 3;  // producer warps 0, 2, 3
// A producer's consecutive chunks are kNProd apart, at most a ring's length: when it waits for
// the release of a stage, the release before that one is already complete (no parity aliasing).
static_assert(kNProd <= kPStages, "producer stride");
constexpr int kPSmem = kPStages * kStageBytes + 1024;

struct UnitInfo {
  TcJob job;
  int mt, m_valid, a_y, nk;
};

// Jobs are read one unit ahead (the load of the next job is in flight while the current unit
// runs), so that no role waits on a global load at a unit boundary.
__device__ __forceinline__ TcJob load_job(const TcJob* __restrict__ jobs, const TcArgs& args, long long u,
                                          long long nunits) {
  return jobs[(u < nunits ? u : nunits - 1) / args.mtiles];
}
__device__ __forceinline__ bool unit_info(const TcJob& job, const TcArgs& args, long long u, UnitInfo& ui) {
  ui.job = job;
  ui.mt = (int)(u % args.mtiles);
  ui.m_valid = min(128, ui.job.m_rows - ui.mt * 128);
  ui.a_y = ui.job.a_y + ui.mt * 128;
  ui.nk = ui.job.nslab * ui.job.nchunk;
  return ui.m_valid > 0 && ui.nk > 0;
}

template <bool CONJ, bool DRAIN>
__global__ void __launch_bounds__(kPThreads, 1)
    k_tc_persist(const __grid_constant__ CUtensorMap amap, const __grid_constant__ CUtensorMap bmap,
                 const TcJob* __restrict__ jobs, const TcArgs args, long long nunits, int* __restrict__ status) {
  constexpr int NB = 2;                             // accumulator buffers
  constexpr uint32_t kBufCols = 128u;
  constexpr uint32_t kImOff = 64u;                  // Im accumulator column offset in a buffer
  constexpr int kHalf = 32;                         // columns per epilogue warpgroup
  constexpr uint32_t kACol = 256u;                  // A stages in tensor memory (64 columns each)
  static_assert(kACol + 64u * kPStages <= 512u && NB * kBufCols <= kACol, "tensor-memory plan");
  extern __shared__ unsigned char dsm_raw[];
  unsigned char* sm = reinterpret_cast<unsigned char*>((reinterpret_cast<uintptr_t>(dsm_raw) + 1023) & ~uintptr_t(1023));
  __shared__ __align__(8) uint64_t bar_full[kPStages], bar_ready[kPStages], bar_empty[kPStages];
  __shared__ __align__(8) uint64_t bar_accf[NB], bar_acce[NB], bar_done;
  __shared__ uint32_t tmem_holder;
  __shared__ volatile int abort_flag;
  __shared__ unsigned long long last_chunk[kPStages];  // 1 + the last chunk issued on each stage (0: none)

  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  if (threadIdx.x == 0) {
    abort_flag = 0;
    for (int s = 0; s < kPStages; ++s) {
      last_chunk[s] = 0ULL;
      mbar_init(su32(&bar_full[s]), 1);
      mbar_init(su32(&bar_ready[s]), 128);
      mbar_init(su32(&bar_empty[s]), 1);
    }
    for (int b = 0; b < NB; ++b) {
      mbar_init(su32(&bar_accf[b]), 1);
      mbar_init(su32(&bar_acce[b]), 256);
    }
    mbar_init(su32(&bar_done), 1);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
  }
  if (warp == 1) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(su32(&tmem_holder)),
                 "r"(512)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  tc_before();
  __syncthreads();
  tc_after();
  const uint32_t tmem = tmem_holder;
  const long long u_step = gridDim.x;

  if (warp == 0 || warp == 2 || warp == 3) {
    if (lane == 0) {
      // ---- producers: every producer walks the whole chunk sequence and issues its own share
      const int prod = warp == 0 ? 0 : warp - 1;
      long long gk = 0;  // chunk counter over all units of this CTA
      UnitInfo ui;
      TcJob nxt = load_job(jobs, args, blockIdx.x, nunits);
      for (long long u = blockIdx.x; u < nunits && !abort_flag; u += u_step) {
        const TcJob cur = nxt;
        nxt = load_job(jobs, args, u + u_step, nunits);
        if (!unit_info(cur, args, u, ui)) continue;
        const TcJob& job = ui.job;
        const int abox = args.a_box;
        const int a_boxes = (ui.m_valid + abox - 1) / abox;
        const uint32_t tx_bytes =
            (uint32_t)(a_boxes * abox * kRowBytes) + (uint32_t)(args.b_rows * kRowBytes * (CONJ ? 1 : 4));
        // the job must describe copies that start on 16-byte boundaries and fit the stage; otherwise
        // nothing is issued, the status records it and the CTA stops
        if (abox <= 0 || 128 % abox != 0 || a_boxes * abox > 128 || args.b_rows != 64 || (job.a_x & 3) ||
            (job.b_x & 3) || job.nchunk < 1 || job.nslab < 1 || job.a_y < 0 || job.b_y < 0) {
          atomicExch(status, (int)DEV_BADJOB);
          abort_flag = 1;
          break;
        }
        bool ok = true;
        for (int kk = 0; kk < ui.nk; ++kk, ++gk) {
          if ((int)(gk % kNProd) != prod) continue;
          const int s = (int)(gk % kPStages);
          const long long round = gk / kPStages;
          if (round > 0 && !mbar_wait(su32(&bar_empty[s]), (uint32_t)((round - 1) & 1), &abort_flag, args.wait_ns)) {
            ok = false;
            break;
          }
          const int slab = kk / job.nchunk, ch = kk - slab * job.nchunk;
          const int ax = job.a_x + kChunkReals * ch, bx = job.b_x + kChunkReals * ch;
          const int az = job.a_z + slab * job.a_dz, bz = job.b_z + slab * job.b_dz;
          const uint32_t full = su32(&bar_full[s]);
          const uint32_t st = su32(sm + s * kStageBytes);
          mbar_expect_tx(full, tx_bytes);
          for (int i = 0; i < a_boxes; ++i)
            tma_load3(st + i * abox * kRowBytes, &amap, ax, ui.a_y + abox * i, az, full);
          if (CONJ)
            tma_load3(st + kABytes, &bmap, bx, job.b_y, bz, full);
          else  // the four variants in one box: [variant][b_rows rows][32 reals]
            tma_load4(st + kABytes, &bmap, bx, job.b_y, 0, bz, full);
          atomicMax(&last_chunk[s], (unsigned long long)(gk + 1));
        }
        if (!ok) break;
      }
    }
  } else if (warp == 1) {
    if (lane == 0) {
      // ---- MMA issuer
      long long gk = 0, gi = 0;  // chunk and accumulator-interval counters over all units
      UnitInfo ui;
      bool ok = true;
      TcJob nxt = load_job(jobs, args, blockIdx.x, nunits);
      for (long long u = blockIdx.x; u < nunits && ok; u += u_step) {
        const TcJob cur = nxt;
        nxt = load_job(jobs, args, u + u_step, nunits);
        if (!unit_info(cur, args, u, ui)) continue;
        // one MMA per product writes Re (columns [0, b_rows)) and Im ([b_rows, 2 b_rows)) together
        const uint32_t idesc = tf32_idesc(2 * args.b_rows);
        const int per = DRAIN ? kDrain : ui.nk;  // chunks per accumulator interval
        uint32_t t_re = 0;
        bool fresh = true;
        for (int kk = 0; kk < ui.nk; ++kk, ++gk) {
          if (kk % per == 0) {
            const int b = (int)(gi % NB);
            if (gi >= NB && !mbar_wait(su32(&bar_acce[b]), (uint32_t)(((gi / NB) - 1) & 1), &abort_flag, args.wait_ns)) {
              ok = false;
              break;
            }
            tc_after();
            t_re = tmem + kBufCols * b;
            fresh = true;
          }
          const int s = (int)(gk % kPStages);
          const long long round = gk / kPStages;
          if (!mbar_wait(su32(&bar_ready[s]), (uint32_t)(round & 1), &abort_flag, args.wait_ns)) {
            ok = false;
            break;
          }
          tc_after();
          const uint32_t base = su32(sm + s * kStageBytes);
#pragma unroll
          for (int sub = 0; sub < kChunkReals / 8; ++sub) {
            const uint32_t o = 32u * sub;  // bytes into the 128-byte rows
            const uint32_t ah = tmem + kACol + 64u * s + 8u * sub, al = ah + 32u;  // A head / tail in TMEM
            const uint32_t bb = base + kABytes + o, vs = (uint32_t)kBVarBytes;
            const uint64_t bh = sw128_desc(bb), bl = sw128_desc(bb + 2 * vs);  // [head | i head], [tail | i tail]
            const uint32_t acc = (fresh && sub == 0) ? 0u : 1u;
            umma_tf32_ta(t_re, al, bh, idesc, acc);
            umma_tf32_ta(t_re, ah, bl, idesc, 1u);
            umma_tf32_ta(t_re, ah, bh, idesc, 1u);
          }
          fresh = false;
          umma_commit(su32(&bar_empty[s]));
          if (kk % per == per - 1 || kk == ui.nk - 1) {
            umma_commit(su32(&bar_accf[gi % NB]));
            ++gi;
          }
        }
      }
      // every MMA issued so far has completed once bar_done fires
      umma_commit(su32(&bar_done));
      mbar_wait(su32(&bar_done), 0, &abort_flag, kDrainNs, false);
    }
  } else if (warp >= 4 && warp < 8) {
    // ---- splitter
    const int t = threadIdx.x - 128;
    const int q = warp & 3, row = 32 * q + lane;  // tensor-memory lane of this thread
    long long gk = 0;
    UnitInfo ui;
    bool ok = true;
    TcJob nxt = load_job(jobs, args, blockIdx.x, nunits);
    for (long long u = blockIdx.x; u < nunits && ok; u += u_step) {
      const TcJob cur = nxt;
      nxt = load_job(jobs, args, u + u_step, nunits);
      if (!unit_info(cur, args, u, ui)) continue;
      for (int kk = 0; kk < ui.nk; ++kk, ++gk) {
        const int s = (int)(gk % kPStages);
        const long long round = gk / kPStages;
        // the outcome of the wait is made warp-uniform before the warp's .sync.aligned tensor-memory
        // stores: lanes that saw the phase complete must not run them without the lanes that gave up
        if (!__all_sync(0xffffffffu, mbar_wait(su32(&bar_full[s]), (uint32_t)(round & 1), &abort_flag, args.wait_ns))) {
          ok = false;
          break;
        }
        unsigned char* st = sm + s * kStageBytes;
        // A: this thread's row (tensor-memory lane) of the 128-byte-swizzled raw tile -> head and tail
        // into the stage's tensor-memory columns (16-byte chunk c of row r sits at c ^ (r & 7)), in
        // two halves of 16 reals
        {
          const float4* rowp = reinterpret_cast<const float4*>(st + row * kRowBytes);
          const uint32_t ta = tmem + ((uint32_t)(32 * q) << 16) + kACol + 64u * s;
#pragma unroll
          for (int hf = 0; hf < 2; ++hf) {
            float x[16], h[16], l[16];
#pragma unroll
            for (int c = 0; c < 4; ++c) {
              const float4 v = rowp[(4 * hf + c) ^ (row & 7)];
              x[4 * c] = v.x; x[4 * c + 1] = v.y; x[4 * c + 2] = v.z; x[4 * c + 3] = v.w;
            }
#pragma unroll
            for (int e = 0; e < 16; ++e) {
              h[e] = tf32_rn(x[e]);
              l[e] = tf32_rn(x[e] - h[e]);
            }
            tmem_st16(ta + 16u * hf, h);
            tmem_st16(ta + 32u + 16u * hf, l);
          }
          tmem_wait_st();
        }
        if (CONJ) {
          constexpr int vstride = kBVarBytes / 16;  // float4s between variants
          float4* b1h = reinterpret_cast<float4*>(st + kABytes);
          float4* b2h = b1h + vstride;
          float4* b1l = b1h + 2 * vstride;
          float4* b2l = b1h + 3 * vstride;
          float4 xb[4];
#pragma unroll
          for (int r = 0; r < 4; ++r)
            if (t + 128 * r < vstride) xb[r] = b1h[t + 128 * r];
#pragma unroll
          for (int r = 0; r < 4; ++r)
            if (t + 128 * r < vstride) {
              const int i = t + 128 * r;
              const float4 h = head4(xb[r]), l = tail4(xb[r], h);
              b1h[i] = h;
              b1l[i] = l;
              b2h[i] = rot4(h);
              b2l[i] = rot4(l);
            }
        }
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
        tc_before();
        mbar_arrive(su32(&bar_ready[s]));
      }
    }
  } else if (warp >= 8) {
    // ---- epilogue: warpgroup (warp - 8) / 4 owns columns [half * kHalf, half * kHalf + kHalf)
    const int half = (warp - 8) >> 2;
    const int q = warp & 3;
    const int row = 32 * q + lane;
    const uint32_t lane_addr = tmem + ((uint32_t)(32 * q) << 16);
    const int c0 = half * kHalf;
    long long gi = 0;
    UnitInfo ui;
    bool ok = true;
    float acc_re[DRAIN ? kHalf : 1], acc_im[DRAIN ? kHalf : 1];
    TcJob nxt = load_job(jobs, args, blockIdx.x, nunits);
    for (long long u = blockIdx.x; u < nunits && ok; u += u_step) {
      const TcJob cur = nxt;
      nxt = load_job(jobs, args, u + u_step, nunits);
      if (!unit_info(cur, args, u, ui)) continue;
      const TcJob& job = ui.job;
      const int n_int = DRAIN ? (ui.nk + kDrain - 1) / kDrain : 1;
      const bool mine = c0 < job.n_mma;  // uniform over the warpgroup
#pragma unroll
      for (int j = 0; j < (DRAIN ? kHalf : 1); ++j) acc_re[j] = acc_im[j] = 0.f;
      const long long R = (long long)ui.a_y + row;
      long long obase, ostride;
      if (args.mode == 0) {
        obase = job.out_off + row;
        ostride = 128;
      } else {
        obase = job.out_off + (R / args.Rs) * args.S1 + (R % args.Rs);
        ostride = args.S2;
      }
      const bool store_row = row < ui.m_valid;
      auto put = [&](int n, float xr, float xi) {
        if (store_row && n < job.n_valid)
          args.out[obase + (long long)n * ostride] =
              make_float2(args.alpha.x * xr - args.alpha.y * xi, args.alpha.x * xi + args.alpha.y * xr);
      };
      for (int it = 0; it < n_int; ++it, ++gi) {
        const int b = (int)(gi % NB);
        // warp-uniform outcome before the .sync.aligned tensor-memory loads (as in the splitter)
        if (!__all_sync(0xffffffffu, mbar_wait(su32(&bar_accf[b]), (uint32_t)((gi / NB) & 1), &abort_flag, args.wait_ns))) {
          ok = false;
          break;
        }
        tc_after();
        const uint32_t base = lane_addr + kBufCols * b + c0;
        if (mine) {
#pragma unroll
          for (int n0 = 0; n0 < kHalf; n0 += 16) {
            if (c0 + n0 < job.n_mma) {
              uint32_t re[16], im[16];
              tmem_ld16(base + n0, re);
              tmem_ld16(base + kImOff + n0, im);
              tmem_wait_ld();
              if (DRAIN) {
#pragma unroll
                for (int j = 0; j < 16; ++j) {
                  acc_re[(n0 + j) & (DRAIN ? kHalf - 1 : 0)] += __uint_as_float(re[j]);
                  acc_im[(n0 + j) & (DRAIN ? kHalf - 1 : 0)] += __uint_as_float(im[j]);
                }
              } else {
#pragma unroll
                for (int j = 0; j < 16; ++j) put(c0 + n0 + j, __uint_as_float(re[j]), __uint_as_float(im[j]));
              }
            }
          }
        }
        tc_before();
        mbar_arrive(su32(&bar_acce[b]));
      }
      if (!ok) break;
      if (DRAIN && mine) {
#pragma unroll
        for (int j = 0; j < kHalf; ++j) put(c0 + j, acc_re[j & (DRAIN ? kHalf - 1 : 0)], acc_im[j & (DRAIN ? kHalf - 1 : 0)]);
      }
    }
  }
  tc_before();
  __syncthreads();
  if (warp == 1) {
    __syncwarp();
    tc_after();
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(512) : "memory");
  }
  if (threadIdx.x == 0) {
    // copies still in flight must land before the CTA exits.  Only the last chunk issued on a stage
    // can be: an earlier one was consumed before its stage could be issued again.
    for (int s = 0; s < kPStages; ++s) {
      const unsigned long long g1 = last_chunk[s];
      if (g1 > 0) mbar_wait(su32(&bar_full[s]), (uint32_t)(((g1 - 1) / kPStages) & 1), &abort_flag, kDrainNs, false);
    }
    // a CTA that stopped records a timeout unless a malformed job was recorded first
    if (abort_flag) atomicCAS(status, (int)DEV_OK, (int)DEV_TIMEOUT);
  }
}

// out[tile] = alpha * sum over the tile's units of their FP32 partial tiles ([n][128] slots),
// summed in FP64 in a fixed order.  One CTA per piece of 256 elements of one tile.
__global__ void k_tc_reduce(const TcTile* __restrict__ tiles, const int2* __restrict__ pieces,
                            const float2* __restrict__ partial, double2* __restrict__ out, double2 alpha,
                            long long slot) {
  const int2 pc = pieces[blockIdx.x];
  const TcTile T = tiles[pc.x];
  const int e = pc.y + threadIdx.x;
  if (e >= T.m_valid * T.n_valid) return;
  const int j = e / T.m_valid, m = e - j * T.m_valid;  // consecutive threads read consecutive rows
  const float2* p = partial + (long long)T.unit_begin * slot + (long long)(T.pn0 + j) * 128 + T.pm0 + m * T.pm_stride;
  const long long us = (long long)T.unit_stride * slot;
  double sx[4] = {0.0, 0.0, 0.0, 0.0}, sy[4] = {0.0, 0.0, 0.0, 0.0};
  int u = 0;
  for (; u + 4 <= T.unit_count; u += 4) {
#pragma unroll
    for (int r = 0; r < 4; ++r) {
      const float2 v = p[(long long)(u + r) * us];
      sx[r] += v.x;
      sy[r] += v.y;
    }
  }
  for (; u < T.unit_count; ++u) {
    const float2 v = p[(long long)u * us];
    sx[0] += v.x;
    sy[0] += v.y;
  }
  const double ax = (sx[0] + sx[1]) + (sx[2] + sx[3]), ay = (sy[0] + sy[1]) + (sy[2] + sy[3]);
  out[T.out_off + (long long)m * T.ld + j] = make_double2(alpha.x * ax - alpha.y * ay, alpha.x * ay + alpha.y * ax);
}

// TF32 head and TF32 tail of a double: head + tail = x to about 2^-22 relative.
__device__ __forceinline__ void split_d(double x, float& h, float& l) {
  h = tf32_rn((float)x);
  l = tf32_rn((float)(x - (double)h));
}

// Dense B operands of the orbital right-multiplies from the packed G(tau) blocks.  For family 0
// B[n][k] = G[k][n] (the multiply D = X G), for family 1 B[n][k] = G[n][k] (D = X G^T).  Layout
// [fam][t][w][variant][n][2 nao] floats, variants (conj B) head, (i conj B) head, (conj B) tail,
// (i conj B) tail: the two heads (and the two tails) form one 128-row B operand whose MMA writes
// Re D and Im D side by side.
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
    // variants in the order (conj B head, i conj B head, conj B tail, i conj B tail)
    split_d(g.x, h, l); base[0] = h; base[2 * vs] = l;  base[vs + 1] = h; base[3 * vs + 1] = l;
    split_d(-g.y, h, l); base[1] = h; base[2 * vs + 1] = l;
    split_d(g.y, h, l); base[vs] = h; base[3 * vs] = l;
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
    base[0] = v[0];        // conj B head
    base[2 * per] = v[1];  // conj B tail
    base[per] = v[2];      // i conj B head
    base[3 * per] = v[3];  // i conj B tail
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

// 3-D map of FP32 data: dims (kreals, rows, slabs), boxes of one chunk (32 reals) x box_rows rows,
// 128-byte swizzle, zero fill outside the tensor.
sgw_status make_map(sgw_ctx* c, CUtensorMap* m, const void* base, long long kreals, long long rows, long long slabs,
                    long long row_bytes, long long slab_bytes, int box_rows = 32) {
  CKS(get_encode(c));
  if ((reinterpret_cast<uintptr_t>(base) & 15) || (row_bytes & 15) || (slab_bytes & 15) || (kreals & 3))
    return c->fail(SGW_ERR_ARG, "tensor-core operand not 16-byte aligned");
  cuuint64_t dims[3] = {(cuuint64_t)kreals, (cuuint64_t)rows, (cuuint64_t)slabs};
  cuuint64_t strides[2] = {(cuuint64_t)row_bytes, (cuuint64_t)slab_bytes};
  cuuint32_t box[3] = {(cuuint32_t)kChunkReals, (cuuint32_t)box_rows, 1};
  cuuint32_t es[3] = {1, 1, 1};
  CUresult r = g_encode(m, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 3, const_cast<void*>(base), dims, strides, box, es,
                        CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                        CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  if (r != CUDA_SUCCESS) return c->fail(SGW_ERR_CUDA, "cuTensorMapEncodeTiled failed (" + std::to_string((int)r) + ")");
  return SGW_OK;
}

// 4-D map of the B operands that carry four variants: dims (kreals, rows, 4, slabs), one box of
// 32 reals x box_rows rows x 4 variants per chunk.
sgw_status make_map4(sgw_ctx* c, CUtensorMap* m, const void* base, long long kreals, long long rows, long long slabs,
                     long long row_bytes, long long var_bytes, long long slab_bytes, int box_rows) {
  CKS(get_encode(c));
  if ((reinterpret_cast<uintptr_t>(base) & 15) || (row_bytes & 15) || (var_bytes & 15) || (slab_bytes & 15) ||
      (kreals & 3))
    return c->fail(SGW_ERR_ARG, "tensor-core operand not 16-byte aligned");
  cuuint64_t dims[4] = {(cuuint64_t)kreals, (cuuint64_t)rows, 4, (cuuint64_t)slabs};
  cuuint64_t strides[3] = {(cuuint64_t)row_bytes, (cuuint64_t)var_bytes, (cuuint64_t)slab_bytes};
  cuuint32_t box[4] = {(cuuint32_t)kChunkReals, (cuuint32_t)box_rows, 4, 1};
  cuuint32_t es[4] = {1, 1, 1, 1};
  CUresult r = g_encode(m, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 4, const_cast<void*>(base), dims, strides, box, es,
                        CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                        CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  if (r != CUDA_SUCCESS) return c->fail(SGW_ERR_CUDA, "cuTensorMapEncodeTiled failed (" + std::to_string((int)r) + ")");
  return SGW_OK;
}

constexpr int kMaxDev = 64;
bool g_attr_done[2][2][kMaxDev] = {};
int g_sms[kMaxDev] = {};

template <bool CONJ, bool DRAIN>
sgw_status launch_gemm(sgw_ctx* c, const CUtensorMap& am, const CUtensorMap& bm, const TcJob* jobs, long long njobs,
                       const TcArgs& a, cudaStream_t st) {
  if (njobs <= 0) return SGW_OK;
  if (a.b_rows != 64) return c->fail(SGW_ERR_ARG, "tensor-core launch: B tiles are 64 rows");
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDev) return c->fail(SGW_ERR_CUDA, "no current device");
  if (!g_attr_done[CONJ][DRAIN][dev]) {
    cudaError_t e = cudaFuncSetAttribute(k_tc_persist<CONJ, DRAIN>, cudaFuncAttributeMaxDynamicSharedMemorySize, kPSmem);
    if (e != cudaSuccess) return c->fail(SGW_ERR_CUDA, std::string("tensor-core kernel attribute: ") + cudaGetErrorString(e));
    if (!g_sms[dev] && cudaDeviceGetAttribute(&g_sms[dev], cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
      return c->fail(SGW_ERR_CUDA, "multiprocessor count");
    g_attr_done[CONJ][DRAIN][dev] = true;
  }
  const long long nunits = njobs * a.mtiles;
  const unsigned grid = (unsigned)std::min<long long>(nunits, g_sms[dev]);
  TcArgs args = a;
  args.wait_ns = c->tc_wait_ns;
  // one CTA per SM (the stage ring fills most of shared memory; all 512 tensor-memory columns)
  k_tc_persist<CONJ, DRAIN><<<grid, kPThreads, kPSmem, st>>>(am, bm, jobs, args, nunits, c->d_status);
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

// Split-K unit length of the Gram reductions (chunks of 32 reals): an environment value fixes it,
// otherwise the autotuner picks one of kUnitCandidates on the first call of a context.
constexpr long long kUnitDefault = 128;
constexpr long long kUnitCandidates[] = {64, 128, 256};
long long unit_override() {
  const char* s = std::getenv("SGW_TC_KCHUNK");
  return s ? std::max(1LL, std::atoll(s)) : 0;
}
bool autotune_enabled() {
  const char* s = std::getenv("SGW_TC_AUTOTUNE");
  return unit_override() == 0 && !(s && std::strcmp(s, "0") == 0);
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

// Gram units over a tau-interleaved A operand: row r of the contraction for local tau tl is row
// r nc + tl of its pair slab, so one 128-row tile holds rpt = 128 / nc values of r for all tau
// values of a chunk against the same B rows.  Rows [r0, r0 + nr) of A against B rows
// [b_y, b_y + ncols) in tiles of 128 x ntile, ordered K range first (the tiles of one K range run
// side by side and share their loads in L2).  Appends the jobs.
// With herm (a Hermitian output whose A rows and B columns index the same range), tiles whose
// rows all lie below their columns are left out; the caller fills them by conjugate transposition.
struct GramTiles {
  long long first;     // first unit (relative to the chunk's first unit)
  int count, stride;   // units per tile, unit stride between the K ranges of one tile
  int mts, nts, rpt, ntile;
  std::vector<int> index;  // [mi * nts + ni]: unit of the tile within a K range, -1 when left out
};
GramTiles gram_interleaved(std::vector<TcJob>& jobs, long long slot0, long long slot, const TcJob& proto, int r0,
                           int nr, int nc, int ncols, int ntile, int nslab, int nchunk, long long unit,
                           bool herm = false) {
  GramTiles g;
  g.rpt = 128 / nc;
  g.ntile = ntile;
  g.mts = (nr + g.rpt - 1) / g.rpt;
  g.nts = (ncols + ntile - 1) / ntile;
  g.index.assign((size_t)g.mts * g.nts, -1);
  int kept = 0;
  for (int mi = 0; mi < g.mts; ++mi)
    for (int ni = 0; ni < g.nts; ++ni)
      if (!(herm && mi * g.rpt >= ntile * (ni + 1))) g.index[(size_t)mi * g.nts + ni] = kept++;
  const std::vector<KRange> kr = split_k(nslab, nchunk, unit);
  g.first = (long long)jobs.size() - slot0;
  g.count = (int)kr.size();
  g.stride = kept;
  for (const KRange& r : kr)
    for (int mi = 0; mi < g.mts; ++mi)
      for (int ni = 0; ni < g.nts; ++ni) {
        if (g.index[(size_t)mi * g.nts + ni] < 0) continue;
        TcJob j = proto;
        j.a_y = (r0 + mi * g.rpt) * nc;
        j.m_rows = std::min(g.rpt, nr - mi * g.rpt) * nc;
        j.b_y = proto.b_y + ntile * ni;
        j.a_z += r.slab0 * proto.a_dz;
        j.b_z += r.slab0 * proto.b_dz;
        j.a_x += kChunkReals * r.c0;
        j.b_x += kChunkReals * r.c0;
        j.nslab = r.nslab;
        j.nchunk = r.nch;
        j.n_valid = std::min(ntile, ncols - ntile * ni);
        j.n_mma = round16(j.n_valid);
        j.out_off = ((long long)jobs.size() - slot0) * slot;
        jobs.push_back(j);
      }
  return g;
}

// Reduction tiles of one output block for local tau tl: A rows [ra0, ra0 + nra) (of the range that
// starts at r0 in gram_interleaved) against B columns [ca0, ca0 + nca), written at out_base (row
// stride ld), split along the tiles they fall in.
void gram_out_tiles(std::vector<TcTile>& tiles, const GramTiles& g, int r0, int nc, int tl, int ra0, int nra,
                    int cb0, int ca0, int nca, long long out_base, int ld) {
  for (int mi = 0; mi < g.mts; ++mi) {
    const int tr0 = r0 + mi * g.rpt, tr1 = tr0 + g.rpt;
    const int a0 = std::max(ra0, tr0), a1 = std::min(ra0 + nra, tr1);
    if (a0 >= a1) continue;
    for (int ni = 0; ni < g.nts; ++ni) {
      const int idx = g.index[(size_t)mi * g.nts + ni];
      if (idx < 0) continue;
      const int tc0 = cb0 + ni * g.ntile, tc1 = tc0 + g.ntile;
      const int b0 = std::max(ca0, tc0), b1 = std::min(ca0 + nca, tc1);
      if (b0 >= b1) continue;
      TcTile t{};
      t.out_off = out_base + (long long)(a0 - ra0) * ld + (b0 - ca0);
      t.ld = ld;
      t.m_valid = a1 - a0;
      t.n_valid = b1 - b0;
      t.pm0 = (a0 - tr0) * nc + tl;
      t.pm_stride = nc;
      t.pn0 = b0 - tc0;
      t.unit_begin = (int)(g.first + idx);
      t.unit_count = g.count;
      t.unit_stride = g.stride;
      tiles.push_back(t);
    }
  }
}

// Launch pieces (tile, first element) of the reduction tiles [t0, t1), 256 elements each.
void reduce_pieces(const std::vector<TcTile>& tiles, long long t0, long long t1, std::vector<int2>& out) {
  for (long long t = t0; t < t1; ++t)
    for (int e = 0; e < tiles[t].m_valid * tiles[t].n_valid; e += 256) out.push_back(make_int2((int)(t - t0), e));
}

int qindex(const sgw_ctx* c, int k1, int k2) {
  const int n1 = c->p.nk[0], n2 = c->p.nk[1], n3 = c->p.nk[2];
  auto iv = [&](int k, int d) { return d == 0 ? k / (n2 * n3) : d == 1 ? (k / n3) % n2 : k % n3; };
  int a = iv(k1, 0) - iv(k2, 0), b = iv(k1, 1) - iv(k2, 1), cc = iv(k1, 2) - iv(k2, 2);
  a = ((a % n1) + n1) % n1; b = ((b % n2) + n2) % n2; cc = ((cc % n3) + n3) % n3;
  return (a * n2 + b) * n3 + cc;
}

// tau values per chunk for at most n per chunk, the chunks balanced over the ntau values
long long balanced_nc(long long nt, long long n) {
  n = std::max(1LL, std::min(n, nt));
  const long long nchunks = (nt + n - 1) / n;
  return (nt + nchunks - 1) / nchunks;
}
long long nc_override() {
  const char* s = std::getenv("SGW_TC_NC");
  return s ? std::max(1LL, std::atoll(s)) : 0;
}

long long tc_nc(const sgw_ctx* c, long long np, long long nt_eff) {
  const long long vs = (long long)c->naux * c->nao * c->nao;
  const double budget = (double)workspace_budget();
  long long nc = (long long)(budget * 0.6 / (2.0 * np * vs * sizeof(float2)));
  nc = std::max(1LL, std::min<long long>({nc, nt_eff, 128LL}));
  const long long nchunks = (nt_eff + nc - 1) / nc;
  return (nt_eff + nchunks - 1) / nchunks;  // balanced chunks
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

static void free_plan_tc(TcPlan*& t) {
  if (!t) return;
  TcPlan& T = *t;
  fr(T.d_vg); fr(T.d_gvg); fr(T.d_pg); fr(T.d_svg); fr(T.d_pvg); fr(T.d_sg); fr(T.d_pr); fr(T.d_sr);
  fr(T.d_prp); fr(T.d_srp);
  fr(T.d_ao_start); fr(T.d_ao_size); fr(T.d_ao_doff); fr(T.d_g_off); fr(T.d_ab_info); fr(T.d_ab_off);
  delete t;
  t = nullptr;
}

void tc_free(sgw_ctx* c) {
  free_plan_tc(c->tc);
  free_plan_tc(c->tc_part);
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

// Gram jobs of P0 for split-K units of `unit` chunks (replaces the previous tables).
static sgw_status build_p0_gram(sgw_ctx* c, TcPlan& T, long long unit) {
  const int Nk = c->Nk, nt = c->nt, nao = c->nao, nc = T.nc_p0, nte = T.nt_eff;
  const long long np = T.pe - T.pb;
  const int nch_g = (2 * nao * nao + kChunkReals - 1) / kChunkReals;
  std::vector<TcJob> pg;
  std::vector<TcTile> pr;
  T.pg_start.assign(nt + 1, 0); T.pr_start.assign(nt + 1, 0);
  // Gram units per tau chunk over the tau-interleaved X: rows (Q, tl) of each pair slab
  std::vector<int2> prp;
  T.prp_start.assign(nt + 1, 0);
  for (int t0 = 0; t0 < nte; t0 += nc) {
    const int t1 = std::min(nte, t0 + nc);
    const long long slot0 = (long long)pg.size(), tile0 = (long long)pr.size();
    for (int t = t0; t < t1; ++t) { T.pg_start[t] = pg.size(); T.pr_start[t] = pr.size(); T.prp_start[t] = prp.size(); }
    for (size_t b = 0; b < c->auxb_off.size(); ++b) {
      const int w = c->auxb_w[b], nb = c->auxb_n[b], s = c->auxb_start[b];
      // the pairs of wedge point w inside the range (none: the block stays zero)
      const long long p0 = std::max(T.pb, (long long)w * Nk), p1 = std::min(T.pe, (long long)(w + 1) * Nk);
      if (p1 <= p0) continue;
      TcJob j{};
      j.a_z = (int)(p0 - T.pb); j.a_dz = 1;  // X slabs are local pairs, V slabs global ones
      j.b_y = s; j.b_z = (int)p0; j.b_dz = 1;
      const GramTiles g = gram_interleaved(pg, slot0, kSlotD, j, s, nb, nc, nb, 64, (int)(p1 - p0), nch_g, unit,
                                           c->herm);
      for (int t = t0; t < t1; ++t)
        gram_out_tiles(pr, g, s, nc, t - t0, s, nb, s, s, nb, (long long)t * c->p_elems + c->auxb_off[b], nb);
    }
    reduce_pieces(pr, tile0, (long long)pr.size(), prp);
  }
  for (int t = nte; t <= nt; ++t) T.prp_start[t] = prp.size();
  CKS(up(c, T.d_prp, prp));
  for (int t = nte; t <= nt; ++t) { T.pg_start[t] = pg.size(); T.pr_start[t] = pr.size(); }
  T.max_units_p0 = 0;
  for (int t0 = 0; t0 < nte; t0 += nc) {
    const int t1 = std::min(nte, t0 + nc);
    T.max_units_p0 = std::max(T.max_units_p0, T.pg_start[t1] - T.pg_start[t0]);
  }
  (void)np;
  CKS(up(c, T.d_pg, pg));
  CKS(up(c, T.d_pr, pr));
  return SGW_OK;
}

static sgw_status build_p0(sgw_ctx* c, TcPlan& T) {
  if (T.built_p0) return SGW_OK;
  CKS(tables_common(c, T));
  const int Nk = c->Nk, nw = c->nwedge, nt = c->nt, nao = c->nao, naux = c->naux, nte = T.nt_eff;
  const long long np = T.pe - T.pb;  // pairs of the range; intermediates are indexed by p - pb
  const int nc = T.nc_req_p0 > 0 ? (int)balanced_nc(nte, T.nc_req_p0) : (int)tc_nc(c, np, nte);
  T.nc_p0 = nc;
  const int rows = naux * nao;
  T.mt_vg = (rows + 127) / 128;
  std::vector<TcJob> vg, gvg;
  T.vg_start.assign(nt + 1, 0); T.gvg_start.assign(nt + 1, 0);
  const int nch_o = (2 * nao + kChunkReals - 1) / kChunkReals;
  // V G jobs of a tau chunk in the order [pair][column tile][tau]: the nc units that read the same
  // V tile for the chunk's tau values run side by side, so V comes from memory once per chunk and
  // from L2 for the other tau values.  G(-tau) Z' jobs read a Z' tile per tau and keep tau order.
  for (int t0 = 0; t0 < nte; t0 += nc) {
    const int t1 = std::min(nte, t0 + nc);
    const long long first = (long long)vg.size();
    for (int t = t0; t < t1; ++t) T.vg_start[t] = first;
    for (long long lp = 0; lp < np; ++lp)
      for (int n0 = 0; n0 < nao; n0 += 64)  // output columns in tiles of 64
        for (int t = t0; t < t1; ++t) {
          const int tl = t - t0;
          const long long p = T.pb + lp;
          const int k2 = c->pair_k2[0][p];
          TcJob j{};
          j.a_y = 0; j.a_z = (int)p; j.b_y = n0;
          j.b_z = (int)(((long long)0 * nt + t) * nw + c->rep[k2]);
          j.a_x = 0; j.b_x = 0; j.nslab = 1; j.nchunk = nch_o; j.a_dz = 0; j.b_dz = 0;
          j.m_rows = rows; j.n_valid = std::min(64, nao - n0); j.n_mma = round16(j.n_valid);
          j.out_off = ((long long)tl * np + lp) * rows * nao + (long long)n0 * nao;  // Z'[A][j][c], column j = n0 + n
          vg.push_back(j);
        }
    for (int t = t0; t < t1; ++t) {
      const int tl = t - t0;
      T.gvg_start[t] = gvg.size();
      for (long long lp = 0; lp < np; ++lp)
        for (int n0 = 0; n0 < nao; n0 += 64) {
          const long long p = T.pb + lp;
          const int k1 = c->pair_k1[0][p];
          TcJob g{};
          g.a_y = 0; g.a_z = (int)((long long)tl * np + lp); g.b_y = n0;
          g.b_z = (int)(((long long)1 * nt + (nt - 1 - t)) * nw + c->rep[k1]);
          g.a_x = 0; g.b_x = 0; g.nslab = 1; g.nchunk = nch_o; g.a_dz = 0; g.b_dz = 0;
          g.m_rows = rows; g.n_valid = std::min(64, nao - n0); g.n_mma = round16(g.n_valid);
          g.out_off = lp * nc * (long long)rows * nao + (long long)tl * nao * nao + (long long)n0 * nao;  // X[p][Q][tl][i][j]
          gvg.push_back(g);
        }
    }
  }
  for (int t = nte; t <= nt; ++t) { T.vg_start[t] = vg.size(); T.gvg_start[t] = gvg.size(); }
  T.unit_p0 = unit_override() ? unit_override() : kUnitDefault;
  if (unit_override()) T.tuned_p0 = true;  // a fixed unit holds for the context's lifetime
  CKS(build_p0_gram(c, T, T.unit_p0));
  T.fl_vg = T.fl_gvg = T.fl_pg = 0;
  for (long long p = T.pb; p < T.pe; ++p) {
    T.fl_vg += 8.0 * naux * nao * (double)c->part_ao[c->rep[c->pair_k2[0][p]]].elems;
    T.fl_gvg += 8.0 * naux * nao * (double)c->part_ao[c->rep[c->pair_k1[0][p]]].elems;
  }
  // with Hermitian blocks the Gram stage needs their upper triangles only
  for (size_t b = 0; b < c->auxb_n.size(); ++b) {
    const int w = c->auxb_w[b];
    const long long npw = std::max(0LL, std::min(T.pe, (long long)(w + 1) * Nk) - std::max(T.pb, (long long)w * Nk));
    T.fl_pg += 8.0 * npw * (double)nao * nao * gram_elems(c, c->auxb_n[b]);
  }
  CKS(up(c, T.d_vg, vg));
  CKS(up(c, T.d_gvg, gvg));
  T.built_p0 = true;
  return SGW_OK;
}

// Gram jobs of Sigma~ for split-K units of `unit` chunks (replaces the previous tables).
static sgw_status build_sigma_gram(sgw_ctx* c, TcPlan& T, long long unit) {
  const int Nk = c->Nk, nw = c->nwedge, nt = c->nt, nao = c->nao, naux = c->naux, nc = T.nc_s;
  const int nch_g = (2 * naux * nao + kChunkReals - 1) / kChunkReals;
  std::vector<TcJob> sg;
  std::vector<TcTile> sr;
  T.sg_start.assign(nt + 1, 0); T.sr_start.assign(nt + 1, 0);
  // Gram units per tau chunk: the whole nao x nao matrix per wedge point over the tau-interleaved X2
  // (rows (i, tl)); the reduction picks the diagonal blocks out of the partial tiles
  std::vector<int2> srp;
  T.srp_start.assign(nt + 1, 0);
  for (int t0 = 0; t0 < nt; t0 += nc) {
    const int t1 = std::min(nt, t0 + nc);
    const long long slot0 = (long long)sg.size(), tile0 = (long long)sr.size();
    for (int t = t0; t < t1; ++t) { T.sg_start[t] = sg.size(); T.sr_start[t] = sr.size(); T.srp_start[t] = srp.size(); }
    for (int w = 0; w < nw; ++w) {
      const long long p0 = std::max(T.pb, (long long)w * Nk), p1 = std::min(T.pe, (long long)(w + 1) * Nk);
      if (p1 <= p0) continue;  // no pairs of this wedge point in the range: its blocks stay zero
      TcJob j{};
      j.a_z = (int)(p0 - T.pb); j.a_dz = 1;  // X2 slabs are local pairs, Vt slabs global ones
      j.b_y = 0; j.b_z = (int)p0; j.b_dz = 1;
      // Hermitian Sigma~ blocks (closed frequency sets): tiles below the diagonal are left out and
      // the blocks' lower triangles filled by conjugate transposition after the reduction
      const GramTiles g = gram_interleaved(sg, slot0, T.slot_s, j, 0, nao, nc, nao, 64, (int)(p1 - p0), nch_g, unit,
                                           c->herm);
      for (int t = t0; t < t1; ++t)
        for (size_t b = 0; b < c->aob_off.size(); ++b) {
          if (c->aob_w[b] != w) continue;
          const int nb = c->aob_n[b], s = c->aob_start[b];
          gram_out_tiles(sr, g, 0, nc, t - t0, s, nb, 0, s, nb, (long long)t * c->g_elems + c->aob_off[b], nb);
        }
    }
    reduce_pieces(sr, tile0, (long long)sr.size(), srp);
  }
  T.srp_start[nt] = srp.size();
  CKS(up(c, T.d_srp, srp));
  T.sg_start[nt] = sg.size(); T.sr_start[nt] = sr.size();
  T.max_units_s = 0;
  for (int t0 = 0; t0 < nt; t0 += nc) {
    const int t1 = std::min(nt, t0 + nc);
    T.max_units_s = std::max(T.max_units_s, T.sg_start[t1] - T.sg_start[t0]);
  }
  CKS(up(c, T.d_sg, sg));
  CKS(up(c, T.d_sr, sr));
  return SGW_OK;
}

static sgw_status build_sigma(sgw_ctx* c, TcPlan& T) {
  if (T.built_sigma) return SGW_OK;
  CKS(tables_common(c, T));
  const int Nk = c->Nk, nw = c->nwedge, nt = c->nt, nao = c->nao, naux = c->naux;
  const long long np = T.pe - T.pb;  // pairs of the range; intermediates are indexed by p - pb
  const int nc = T.nc_req_s > 0 ? (int)balanced_nc(nt, T.nc_req_s) : (int)tc_nc(c, np, nt);
  T.nc_s = nc;
  T.slot_s = kSlotD;
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
    kmax = std::max(kmax, (d + 2 * nb + kChunkReals - 1) / kChunkReals * kChunkReals);
    wblocks[c->auxb_w[b]].push_back(b);
  }
  T.pt_rows = rmax;
  T.pt_k = kmax;
  CKS(up(c, T.d_ab_info, info));
  CKS(up(c, T.d_ab_off, boff));
  const int rows_v = nao * naux, rows_x = nao * nao;
  T.mt_svg = (rows_v + 127) / 128;
  T.mt_pvg = (rows_x + 127) / 128;
  std::vector<TcJob> svg, pvg;
  T.svg_start.assign(nt + 1, 0); T.pvg_start.assign(nt + 1, 0);
  const int nch_o = (2 * nao + kChunkReals - 1) / kChunkReals;
  // Vt G jobs in the order [pair][column tile][tau] within a tau chunk (Vt read once per chunk, as
  // for P0); P^T X1 jobs read an X1 tile per tau and keep tau order
  for (int t0 = 0; t0 < nt; t0 += nc) {
    const int t1 = std::min(nt, t0 + nc);
    const long long first = (long long)svg.size();
    for (int t = t0; t < t1; ++t) T.svg_start[t] = first;
    for (long long lp = 0; lp < np; ++lp)
      for (int n0 = 0; n0 < nao; n0 += 64)  // output columns in tiles of 64
        for (int t = t0; t < t1; ++t) {
          const int tl = t - t0;
          const long long p = T.pb + lp;
          const int k2 = c->pair_k2[1][p];
          TcJob j{};
          j.a_y = 0; j.a_z = (int)p; j.b_y = n0;
          j.b_z = (int)((long long)t * nw + c->rep[k2]);
          j.nslab = 1; j.nchunk = nch_o;
          j.m_rows = rows_v; j.n_valid = std::min(64, nao - n0); j.n_mma = round16(j.n_valid);
          j.out_off = ((long long)tl * np + lp) * vs + (long long)n0 * naux;  // X1T[i][b][A], column b = n0 + n
          svg.push_back(j);
        }
    for (int t = t0; t < t1; ++t) {
      const int tl = t - t0;
      T.pvg_start[t] = pvg.size();
      for (long long lp = 0; lp < np; ++lp) {
        const long long p = T.pb + lp;
        const int k1 = c->pair_k1[1][p], k2 = c->pair_k2[1][p];
        const int wq = c->rep[qindex(c, k1, k2)];
        for (int b : wblocks[wq]) {
          const int s = info[3 * b], nb = info[3 * b + 1], d = info[3 * b + 2];
          for (int n0 = 0; n0 < nb; n0 += 64) {
            TcJob v{};
            v.a_y = 0; v.a_z = (int)((long long)tl * np + lp);
            v.a_x = 2 * s - d;
            v.b_y = n0; v.b_z = tl * ninst + b;
            v.b_x = 0;
            v.nslab = 1; v.nchunk = (d + 2 * nb + kChunkReals - 1) / kChunkReals;
            v.m_rows = rows_x; v.n_valid = std::min(64, nb - n0); v.n_mma = round16(v.n_valid);
            v.out_off = lp * nc * vs + (long long)tl * naux * nao + (long long)(s + n0) * nao;  // X2[p][i][tl][A'][b]
            pvg.push_back(v);
          }
        }
      }
    }
  }
  T.svg_start[nt] = svg.size(); T.pvg_start[nt] = pvg.size();
  T.unit_s = unit_override() ? unit_override() : kUnitDefault;
  if (unit_override()) T.tuned_s = true;
  CKS(build_sigma_gram(c, T, T.unit_s));
  T.fl_svg = T.fl_pvg = T.fl_sg = 0;
  for (long long p = T.pb; p < T.pe; ++p) {
    const int k1 = c->pair_k1[1][p], k2 = c->pair_k2[1][p];
    T.fl_svg += 8.0 * naux * nao * (double)c->part_ao[c->rep[k2]].elems;
    T.fl_pvg += 8.0 * nao * nao * (double)c->part_aux[c->rep[qindex(c, k1, k2)]].elems;
  }
  // with Hermitian blocks the Gram stage needs their upper triangles only
  for (size_t b = 0; b < c->aob_n.size(); ++b) {
    const int w = c->aob_w[b];
    const long long npw = std::max(0LL, std::min(T.pe, (long long)(w + 1) * Nk) - std::max(T.pb, (long long)w * Nk));
    T.fl_sg += 8.0 * npw * (double)naux * nao * gram_elems(c, c->aob_n[b]);
  }
  CKS(up(c, T.d_svg, svg));
  CKS(up(c, T.d_pvg, pvg));
  T.built_sigma = true;
  return SGW_OK;
}

// The plan of the pair range [pb, pe): the whole pair list has its own; one partial range is kept
// (a rank of a partitioned run asks for the same range every time).
static TcPlan& plan_for(sgw_ctx* c, long long pb, long long pe) {
  const bool whole = pb == 0 && pe == (long long)c->nwedge * c->Nk;
  TcPlan*& t = whole ? c->tc : c->tc_part;
  if (t && (t->pb != pb || t->pe != pe)) free_plan_tc(t);
  if (!t) {
    t = new TcPlan();
    t->pb = pb;
    t->pe = pe;
    t->nt_eff = p0_tau_count(c, pb, pe);
  }
  return *t;
}

static bool capturing(cudaStream_t st) {
  cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
  return cudaStreamIsCapturing(st, &cs) != cudaSuccess || cs != cudaStreamCaptureStatusNone;
}

// Autotuner of the split-K unit length of a Gram reduction: build the jobs for each candidate,
// time the launch of the first tau chunk (Gram + FP64 sum of the partial tiles, second of two
// runs, CUDA events on the launching stream) and keep the fastest.  Runs once per context, on
// the first call outside a stream capture.
template <class Build, class Launch>
static sgw_status tune_unit(sgw_ctx* c, cudaStream_t st, const char* what, long long& unit, Build&& build,
                            Launch&& launch) {
  cudaEvent_t a, b;
  if (cudaEventCreate(&a) != cudaSuccess || cudaEventCreate(&b) != cudaSuccess)
    return c->fail(SGW_ERR_CUDA, "autotuner events");
  long long best_unit = unit;
  float best = 1e30f;
  for (long long cand : kUnitCandidates) {
    CKS(build(cand));
    float ms = 0.f;
    for (int rep = 0; rep < 2; ++rep) {
      cudaEventRecord(a, st);
      CKS(launch());
      cudaEventRecord(b, st);
      if (cudaEventSynchronize(b) != cudaSuccess) return c->fail(SGW_ERR_CUDA, "autotuner timing");
      cudaEventElapsedTime(&ms, a, b);
    }
    if (ms < best) {
      best = ms;
      best_unit = cand;
    }
  }
  cudaEventDestroy(a);
  cudaEventDestroy(b);
  unit = best_unit;
  CKS(build(unit));
  const char* v = std::getenv("SGW_VERBOSE");
  if (v && v[0] == '1') std::fprintf(stderr, "sgw autotune: %s split-K unit %lld chunks (%.3f ms)\n", what, unit, best);
  return SGW_OK;
}

// The P0 chain over the plan's tau chunks.  With trial_ms, only the first chunk runs, twice, and
// the time of the second run (ms) is returned there (the tau-chunk autotuner).
static sgw_status p0_run(sgw_ctx* c, TcPlan& T, const double2* G, double2* out, cudaStream_t st, float* trial_ms) {
  const int nt = c->nt, nw = c->nwedge, nao = c->nao, naux = c->naux, Nk = c->Nk, nc = T.nc_p0;
  // np: pairs of the range (intermediate slabs); npg: the whole pair list (V slabs)
  const long long np = T.pe - T.pb, npg = (long long)nw * Nk, vs = (long long)naux * nao * nao;
  const long long inter = (long long)nc * np * vs;  // complex64 elements
  const long long gop = 2LL * nt * nw * 4 * nao * 2 * nao;  // floats
  const bool tune = !T.tuned_p0 && autotune_enabled() && !capturing(st) && !trial_ms;
  long long max_units = T.max_units_p0;
  if (tune) {  // partial tiles for the candidate with the most units
    for (long long cand : kUnitCandidates) {
      CKS(build_p0_gram(c, T, cand));
      max_units = std::max(max_units, T.max_units_p0);
    }
    CKS(build_p0_gram(c, T, T.unit_p0));
  }
  const long long b_z = al256(inter * 8), b_x = al256(inter * 8), b_g = al256(gop * 4),
                  b_p = al256(max_units * kSlotD * 8);
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
  CKS(make_map(c, &mV, c->d_V32[0], 2 * nao, rows, npg, 8LL * nao, vs * 8, 128));
  CKS(make_map(c, &mZ, Zp, 2 * nao, rows, (long long)nc * np, 8LL * nao, vs * 8, 128));
  CKS(make_map4(c, &mG, Gop, 2 * nao, nao, 2LL * nt * nw, 8LL * nao, 8LL * nao * nao, 32LL * nao * nao, 64));
  // Gram operands: rows Q, contracted (i, j) re/im
  CUtensorMap mXg, mVg;
  CKS(make_map(c, &mXg, X, 2LL * nao * nao, (long long)naux * nc, np, 8LL * nao * nao, (long long)nc * vs * 8, 32));
  CKS(make_map(c, &mVg, c->d_V32[0], 2LL * nao * nao, naux, npg, 8LL * nao * nao, vs * 8, 64));
  const double alpha = c->p.loop_sign * (double)c->p.spin_factor / c->Nk;
  const int nte = T.nt_eff;  // tau values contracted (the reflection gives the rest)
  const int t_end = trial_ms ? std::min(nte, nc) : nte, reps = trial_ms ? 2 : 1;
  cudaEvent_t ea = nullptr, eb = nullptr;
  if (trial_ms && (cudaEventCreate(&ea) != cudaSuccess || cudaEventCreate(&eb) != cudaSuccess))
    return c->fail(SGW_ERR_CUDA, "autotuner events");
  for (int rep = 0; rep < reps; ++rep) {
  if (trial_ms && rep == reps - 1) cudaEventRecord(ea, st);
  for (int t0 = 0; t0 < t_end; t0 += nc) {
    const int t1 = std::min(nte, t0 + nc), ntc = t1 - t0;
    TcArgs a{};
    a.a_box = 128;
    a.b_rows = 64;
    a.mtiles = T.mt_vg; a.mode = 1; a.Rs = nao; a.S1 = (long long)nao * nao; a.S2 = nao;
    a.alpha = make_float2(1.f, 0.f); a.out = Zp;
    // Z'[A][j][c] = sum_d V[A][c][d] G^{k+q}(tau)[d][j]
    sgw_status s1 = SGW_OK, s2 = SGW_OK, s3 = SGW_OK;
    run(c, "p0_vg_tc", T.fl_vg * ntc, 1, st, [&] {
      s1 = launch_gemm<false, false>(c, mV, mG, T.d_vg + T.vg_start[t0], T.vg_start[t1] - T.vg_start[t0], a, st);
    });
    CKS(s1);
    // X[A][tl][i][j] = sum_c G^k(-tau)[i][c] Z'[A][j][c],  G(-tau_j) = -G(tau_{n-1-j})
    a.alpha = make_float2(-1.f, 0.f); a.out = X;
    a.S1 = (long long)nc * nao * nao;
    run(c, "p0_gvg_tc", T.fl_gvg * ntc, 1, st, [&] {
      s2 = launch_gemm<false, false>(c, mZ, mG, T.d_gvg + T.gvg_start[t0], T.gvg_start[t1] - T.gvg_start[t0], a, st);
    });
    CKS(s2);
    // P0 block tiles: sum over k and (i, j) of X[Q][(i,j)] conj(V[Q'][(i,j)])
    TcArgs g{};
    g.a_box = 32;
    g.b_rows = 64;
    g.mtiles = 1; g.mode = 0; g.Rs = 1; g.alpha = make_float2(1.f, 0.f); g.out = part;
    auto gemm = [&]() {
      return launch_gemm<true, true>(c, mXg, mVg, T.d_pg + T.pg_start[t0], T.pg_start[t1] - T.pg_start[t0], g, st);
    };
    auto reduce = [&]() {
      const long long r0 = T.pr_start[t0], q0 = T.prp_start[t0], q1 = T.prp_start[t1];
      if (q1 > q0)
        k_tc_reduce<<<(unsigned)(q1 - q0), 256, 0, st>>>(T.d_pr + r0, T.d_prp + q0, part, out, make_double2(alpha, 0.0),
                                                         kSlotD);
    };
    if (tune && t0 == 0) {
      auto both = [&]() -> sgw_status {
        CKS(gemm());
        reduce();
        return SGW_OK;
      };
      CKS(tune_unit(c, st, "P0", T.unit_p0, [&](long long u) { return build_p0_gram(c, T, u); }, both));
      T.tuned_p0 = true;
    }
    run(c, "p0_gram_tc", T.fl_pg * ntc, 1, st, [&] { s3 = gemm(); });
    CKS(s3);
    run(c, "gram_reduce", 0.0, 1, st, reduce);
  }
  }
  if (trial_ms) {
    cudaEventRecord(eb, st);
    const bool ok = cudaEventSynchronize(eb) == cudaSuccess && cudaEventElapsedTime(trial_ms, ea, eb) == cudaSuccess;
    cudaEventDestroy(ea);
    cudaEventDestroy(eb);
    return ok ? SGW_OK : c->fail(SGW_ERR_CUDA, "autotuner timing");
  }
  if (tune) T.tuned_p0 = true;
  return p0_complete(c, out, nte, st);
}

// Candidate tau chunks of the autotuner: the largest the workspace allows, about half and about a
// quarter of it (distinct, balanced over the tau values), largest first.
static std::vector<int> nc_candidates(long long nt, long long ncmax) {
  std::vector<int> out;
  for (long long d : {1LL, 2LL, 4LL}) {
    const int v = (int)balanced_nc(nt, (ncmax + d - 1) / d);
    if (std::find(out.begin(), out.end(), v) == out.end()) out.push_back(v);
  }
  return out;
}

// Tau-chunk autotuner: the chunk sets the shape of the Gram tiles (128 rows = 128 / nc auxiliary
// rows x nc tau values against the same V rows), how often V is read and the number of launches.
// On a context's first call outside a stream capture each candidate is built and the first chunk
// of the chain timed (second of two runs); the fastest per tau value is kept.  SGW_TC_NC fixes it.
template <class Build, class Run>
static sgw_status tune_nc(sgw_ctx* c, long long nt, long long ncmax, int& req, bool& built, const char* what,
                          Build&& build, Run&& runone) {
  const std::vector<int> cands = nc_candidates(nt, ncmax);
  if (cands.size() < 2) return SGW_OK;
  float best = 1e30f;
  int best_nc = cands[0];
  for (int cand : cands) {
    req = cand;
    built = false;
    CKS(build());
    float ms = 0.f;
    CKS(runone(&ms));
    if (ms / cand < best) {
      best = ms / cand;
      best_nc = cand;
    }
  }
  req = best_nc;
  built = false;
  const char* v = std::getenv("SGW_VERBOSE");
  if (v && v[0] == '1')
    std::fprintf(stderr, "sgw autotune: %s tau chunk %d (%.4f ms per tau value)\n", what, best_nc, best);
  return SGW_OK;
}

sgw_status tc_polarization(sgw_ctx* c, const double2* G, double2* out, long long pb, long long pe, cudaStream_t st) {
  TcPlan& T = plan_for(c, pb, pe);
  if (!T.tuned_nc_p0) {
    if (nc_override()) {
      T.nc_req_p0 = (int)nc_override();
      T.built_p0 = false;
      T.tuned_nc_p0 = true;
    } else if (autotune_enabled() && !capturing(st)) {
      CKS(tune_nc(c, T.nt_eff, tc_nc(c, T.pe - T.pb, T.nt_eff), T.nc_req_p0, T.built_p0, "P0", [&] { return build_p0(c, T); },
                  [&](float* ms) { return p0_run(c, T, G, out, st, ms); }));
      T.tuned_nc_p0 = true;
    }
  }
  CKS(build_p0(c, T));
  return p0_run(c, T, G, out, st, nullptr);
}

static sgw_status s_run(sgw_ctx* c, TcPlan& T, const double2* G, const double2* P, double2* out, cudaStream_t st,
                        float* trial_ms) {
  const int nt = c->nt, nw = c->nwedge, nao = c->nao, naux = c->naux, Nk = c->Nk, nc = T.nc_s;
  const long long np = T.pe - T.pb, npg = (long long)nw * Nk, vs = (long long)naux * nao * nao;
  const long long inter = (long long)nc * np * vs;
  const long long gop = 1LL * nt * nw * 4 * nao * 2 * nao;
  const long long pop = (long long)nc * T.ninst * 4 * T.pt_rows * T.pt_k;
  const bool tune = !T.tuned_s && autotune_enabled() && !capturing(st) && !trial_ms;
  long long max_units = T.max_units_s;
  if (tune) {  // partial tiles for the candidate with the most units
    for (long long cand : kUnitCandidates) {
      CKS(build_sigma_gram(c, T, cand));
      max_units = std::max(max_units, T.max_units_s);
    }
    CKS(build_sigma_gram(c, T, T.unit_s));
  }
  const long long b_1 = al256(inter * 8), b_2 = al256(inter * 8), b_g = al256(gop * 4), b_pp = al256(pop * 4),
                  b_p = al256(max_units * T.slot_s * 8);
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
  CKS(make_map(c, &mVt, c->d_V32[1], 2 * nao, rows_v, npg, 8LL * nao, vs * 8, 128));
  CKS(make_map4(c, &mG, Gop, 2 * nao, nao, 1LL * nt * nw, 8LL * nao, 8LL * nao * nao, 32LL * nao * nao, 64));
  CKS(make_map(c, &mX1, X1, 2LL * naux, (long long)nao * nao, (long long)nc * np, 8LL * naux, vs * 8, 128));
  CKS(make_map4(c, &mP, Pop, T.pt_k, T.pt_rows, (long long)nc * T.ninst, 4LL * T.pt_k, 4LL * T.pt_k * T.pt_rows,
                16LL * T.pt_k * T.pt_rows, 64));
  CKS(make_map(c, &mX2g, X2, 2LL * naux * nao, (long long)nao * nc, np, 8LL * naux * nao, (long long)nc * vs * 8, 32));
  CKS(make_map(c, &mVtg, c->d_V32[1], 2LL * naux * nao, nao, npg, 8LL * naux * nao, vs * 8, 64));
  const int t_end = trial_ms ? std::min(nt, nc) : nt, reps = trial_ms ? 2 : 1;
  cudaEvent_t ea = nullptr, eb = nullptr;
  if (trial_ms && (cudaEventCreate(&ea) != cudaSuccess || cudaEventCreate(&eb) != cudaSuccess))
    return c->fail(SGW_ERR_CUDA, "autotuner events");
  for (int rep = 0; rep < reps; ++rep) {
  if (trial_ms && rep == reps - 1) cudaEventRecord(ea, st);
  for (int t0 = 0; t0 < t_end; t0 += nc) {
    const int t1 = std::min(nt, t0 + nc), ntc = t1 - t0;
    run(c, "tc_prep", 0.0, 1, st, [&] {
      k_tc_p_operands<<<gridn((long long)ntc * T.ninst * T.pt_rows * T.pt_k, 256), 256, 0, st>>>(
          P, c->p_elems, t0, ntc, T.d_ab_info, T.d_ab_off, T.ninst, T.pt_rows, T.pt_k, Pop);
    });
    sgw_status s1 = SGW_OK, s2 = SGW_OK, s3 = SGW_OK;
    // X1T[i][b][A] = sum_a V[A][i][a] G^{k2}(tau)[a][b]
    TcArgs a{};
    a.a_box = 128;
    a.b_rows = 64;
    a.mtiles = T.mt_svg; a.mode = 1; a.Rs = naux; a.S1 = (long long)nao * naux; a.S2 = naux;
    a.alpha = make_float2(1.f, 0.f); a.out = X1;
    run(c, "sigma_vg_tc", T.fl_svg * ntc, 1, st, [&] {
      s1 = launch_gemm<false, false>(c, mVt, mG, T.d_svg + T.svg_start[t0], T.svg_start[t1] - T.svg_start[t0], a, st);
    });
    CKS(s1);
    // X2[i][tl][A'][b] = sum_A P^q(tau)[A][A'] X1T[i][b][A]
    TcArgs b{};
    b.a_box = 128;
    b.b_rows = 64;
    b.mtiles = T.mt_pvg; b.mode = 1; b.Rs = nao; b.S1 = (long long)nc * naux * nao; b.S2 = nao;
    b.alpha = make_float2(1.f, 0.f); b.out = X2;
    run(c, "sigma_pvg_tc", T.fl_pvg * ntc, 1, st, [&] {
      s2 = launch_gemm<false, true>(c, mX1, mP, T.d_pvg + T.pvg_start[t0], T.pvg_start[t1] - T.pvg_start[t0], b, st);
    });
    CKS(s2);
    // Sigma tiles: sum over k2 and (A', b) of X2[(i,tl)][(A',b)] conj(Vt[i'][(A',b)])
    TcArgs g{};
    g.a_box = 32;
    g.b_rows = 64;
    g.mtiles = 1; g.mode = 0; g.Rs = 1; g.alpha = make_float2(1.f, 0.f); g.out = part;
    auto gemm = [&]() {
      return launch_gemm<true, true>(c, mX2g, mVtg, T.d_sg + T.sg_start[t0], T.sg_start[t1] - T.sg_start[t0], g, st);
    };
    auto reduce = [&]() {
      const long long r0 = T.sr_start[t0], q0 = T.srp_start[t0], q1 = T.srp_start[t1];
      if (q1 > q0)
        k_tc_reduce<<<(unsigned)(q1 - q0), 256, 0, st>>>(T.d_sr + r0, T.d_srp + q0, part, out,
                                                         make_double2(-1.0 / c->Nk, 0.0), T.slot_s);
    };
    if (tune && t0 == 0) {
      auto both = [&]() -> sgw_status {
        CKS(gemm());
        reduce();
        return SGW_OK;
      };
      CKS(tune_unit(c, st, "Sigma", T.unit_s, [&](long long u) { return build_sigma_gram(c, T, u); }, both));
      T.tuned_s = true;
    }
    run(c, "sigma_gram_tc", T.fl_sg * ntc, 1, st, [&] { s3 = gemm(); });
    CKS(s3);
    run(c, "gram_reduce", 0.0, 1, st, reduce);
  }
  }
  if (trial_ms) {
    cudaEventRecord(eb, st);
    const bool ok = cudaEventSynchronize(eb) == cudaSuccess && cudaEventElapsedTime(trial_ms, ea, eb) == cudaSuccess;
    cudaEventDestroy(ea);
    cudaEventDestroy(eb);
    return ok ? SGW_OK : c->fail(SGW_ERR_CUDA, "autotuner timing");
  }
  if (tune) T.tuned_s = true;
  return lower_from_upper(c, 0, out, st);
}

sgw_status tc_self_energy(sgw_ctx* c, const double2* G, const double2* P, double2* out, long long pb, long long pe,
                          cudaStream_t st) {
  TcPlan& T = plan_for(c, pb, pe);
  if (!T.tuned_nc_s) {
    if (nc_override()) {
      T.nc_req_s = (int)nc_override();
      T.built_sigma = false;
      T.tuned_nc_s = true;
    } else if (autotune_enabled() && !capturing(st)) {
      CKS(tune_nc(c, c->nt, tc_nc(c, T.pe - T.pb, c->nt), T.nc_req_s, T.built_sigma, "Sigma",
                  [&] { return build_sigma(c, T); }, [&](float* ms) { return s_run(c, T, G, P, out, st, ms); }));
      T.tuned_nc_s = true;
    }
  }
  CKS(build_sigma(c, T));
  return s_run(c, T, G, P, out, st, nullptr);
}

}  // namespace sgw
