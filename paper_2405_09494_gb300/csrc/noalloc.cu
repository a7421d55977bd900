// sgw_screened_interaction_noalloc: the screened-interaction step with its scratch in a
// fixed, file-scope device array, for callers that must not allocate device memory when they
// call in (for example code that runs while another component is capturing a CUDA graph,
// where cudaMalloc is not permitted, or a host application that fixes its device memory
// budget at start-up and forbids allocations afterwards).
#include <cmath>
#include <cstring>
#include <mutex>

#include "sgw_internal.h"

using namespace sgw;

namespace {

// Scratch of the entry point: the P0(i Omega) and P(i Omega) frequency series, 4 Mi complex
// numbers (64 MiB).  It is part of the library image, so every GPU that loads the library holds
// it until the process exits; all calls share it.
constexpr long long kNoAllocElems = 4LL << 20;
static __device__ __align__(256) double2 g_noalloc_scratch[kNoAllocElems];

// Device address of the scratch, looked up once per device (host code may not use the
// symbol itself: on the host it only names a stand-in, not device memory).
constexpr int kMaxDevices = 64;
std::mutex g_mu;
void* g_ptr[kMaxDevices] = {nullptr};

sgw_status scratch_address(sgw_ctx* c, double2** out) {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return c->fail(SGW_ERR_CUDA, std::string("cudaGetDevice: ") + cudaGetErrorString(e));
  // the context's tables and the scratch must be on one device: the array's address is per device
  if (dev != c->device)
    return c->fail(SGW_ERR_STATE, "sgw_screened_interaction_noalloc: the current device (" + std::to_string(dev) +
                                      ") is not the context's (" + std::to_string(c->device) + ")");
  if (dev < 0 || dev >= kMaxDevices) return c->fail(SGW_ERR_ARG, "device ordinal out of range");
  std::lock_guard<std::mutex> lock(g_mu);
  if (g_ptr[dev] == nullptr) {
    void* p = nullptr;
    e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
    if (e != cudaSuccess || p == nullptr)
      return c->fail(SGW_ERR_CUDA, std::string("cudaGetSymbolAddress of the fixed scratch: ") + cudaGetErrorString(e));
    g_ptr[dev] = p;
  }
  *out = static_cast<double2*>(g_ptr[dev]);
  return SGW_OK;
}

}  // namespace

extern "C" SGW_API sgw_status sgw_screened_interaction_noalloc(sgw_ctx* c, const void* P0_tau, void* P_tau,
                                                               sgw_stream stream) {
  if (!c) return SGW_ERR_ARG;
  if (!c->built) return c->fail(SGW_ERR_STATE, "sgw_build_irrep_basis has not been called");
  if (!P0_tau || !P_tau) return c->fail(SGW_ERR_ARG, "null series pointer");
  if (!c->tables)
    return c->fail(SGW_ERR_STATE,
                   "sgw_screened_interaction_noalloc reuses the launch tables that sgw_screened_interaction builds: "
                   "call sgw_screened_interaction once on this context first");
  const long long pe = c->p_elems;
  const long long need = 2LL * c->nwb * pe;
  if (need > kNoAllocElems)
    return c->fail(SGW_ERR_ARG, "sgw_screened_interaction_noalloc: 2 * nw_b * p_elems = " + std::to_string(need) +
                                    " complex numbers exceed the fixed scratch of " + std::to_string(kNoAllocElems) +
                                    " (64 MiB); use sgw_screened_interaction");
  if (c->max_aux_block > 90)
    return c->fail(SGW_ERR_ARG,
                   "sgw_screened_interaction_noalloc: auxiliary blocks above 90 need per-block scratch; use "
                   "sgw_screened_interaction");
  double2* scr = nullptr;
  {
    sgw_status s = scratch_address(c, &scr);
    if (s != SGW_OK) return s;
  }
  cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
  double2* P0w = scr;                      // [nw_b][p_elems], fully overwritten below
  double2* Pw = scr + (size_t)c->nwb * pe;  // [nw_b][p_elems], fully overwritten below
  const double2 one = make_double2(1.0, 0.0);
  // the launch accounting of sgw_screened_interaction (it records CUDA events only, when profiling
  // is on, and allocates no device memory)
  const double flt = 8.0 * c->nwb * (double)c->nt * pe;
  double flw = 0;
  for (size_t b = 0; b < c->auxb_n.size(); ++b) flw += 8.0 * c->nwb * std::pow((double)c->auxb_n[b], 3);
  run(c, "ft", flt, 1, st, [&] {
    series_map(c->d_TB, c->nwb, c->nt, static_cast<const double2*>(P0_tau), pe, P0w, pe, pe, one, 0, st);
  });
  run(c, "w_solve", flw, 1, st, [&] {
    invert_plan(INV_W, c->w_plan, P0w, nullptr, nullptr, nullptr, 0.0, nullptr, nullptr, Pw, nullptr, nullptr,
                c->d_status, st);
  });
  run(c, "ft", flt, 1, st, [&] {
    series_map(c->d_TBbar, c->nt, c->nwb, Pw, pe, static_cast<double2*>(P_tau), pe, pe, one, 0, st);
  });
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return c->fail(SGW_ERR_CUDA, std::string("launch: ") + cudaGetErrorString(e));
  return SGW_OK;
}
