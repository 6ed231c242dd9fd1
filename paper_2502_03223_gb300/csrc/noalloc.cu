// Allocation-free variant of the hydro right-hand side of one level.
//
// Some callers cannot call cudaMalloc: code that embeds this library inside
// a host application whose memory pool already owns the device (a framework
// caching allocator, a pre-reserved simulation arena), or that runs where
// allocation is not allowed or its latency is not acceptable.  For them this
// entry point computes the same face fluxes and flux divergence with sources
// as the hydro part of sacra_rk_stage, with its scratch (the face fluxes) in
// a file-scope static device array instead of an arena.  The caller passes
// inputs and outputs only; nothing is allocated or freed.
#include <string.h>

#include "kernels.h"

using namespace sacra;

namespace {

constexpr size_t kMaxPlane = SACRA_NOALLOC_MAX_PLANE;   // padded plane of at most 256 x 256 interior cells
constexpr size_t kScratchDoubles = 2 * NCONS * kMaxPlane + 32;   // x and z face fluxes + a counter

// Shared by every call on a device and kept between calls; every GPU that
// loads the library holds it (about 5.9 MB) until the process exits.  The
// last word counts HLLC -> TVDLF fallbacks; this entry point does not report
// it (the kernels need somewhere to count).
static __device__ __align__(256) double g_scratch[kScratchDoubles];

}  // namespace

extern "C" sacra_status sacra_hydro_rhs_noalloc(const sacra_params *p, int level, const double *state,
                                                const double *prims, double *rhs_out, void *cuda_stream) {
  if (!p || !state || !prims || !rhs_out) return SACRA_ERR_ARG;
  if (level < 0 || level >= p->n_levels || p->nx < 8 || p->nz < 4) return SACRA_ERR_ARG;
  if (p->geometry != SACRA_PLANAR && p->geometry != SACRA_CYLINDRICAL) return SACRA_ERR_ARG;
  if (p->solver != SACRA_HLLC && p->solver != SACRA_TVDLF) return SACRA_ERR_ARG;
  if (!(p->dx0 > 0) || !(p->dz0 > 0) || !(p->Gamma_th > 1.0)) return SACRA_ERR_ARG;
  if (p->n_pieces > 1) return SACRA_ERR_ARG;          // the piece table needs the context's device memory
  if (p->eos_adiabatic && !(p->K > 0.0)) return SACRA_ERR_ARG;
  if (p->precision & ~SACRA_MIXED) return SACRA_ERR_ARG;
  const size_t px = (size_t)p->nx + 2 * GH, pz = (size_t)p->nz + 2 * GH;
  if (px * pz > kMaxPlane) return SACRA_ERR_ARG;    // beyond the static scratch

  // An error the calling thread left unread belongs to earlier work: report
  // it without clearing it or launching anything, so that the check after
  // the launches below sees this call's launches only.
  if (cudaPeekAtLastError() != cudaSuccess) return SACRA_ERR_CUDA;

  // The device address of the static array on the current device (its
  // host-side name is only a stand-in).  Looked up on every call: the lookup
  // allocates nothing, and a context torn down and created again (after
  // cudaDeviceReset, say) reloads the module at another address.  The first
  // call on a device loads the module, so make it before any stream capture.
  double *scratch = nullptr;
  if (cudaGetSymbolAddress((void **)&scratch, g_scratch) != cudaSuccess || !scratch) {
    cudaGetLastError();
    return SACRA_ERR_CUDA;
  }

  DevParams d;
  fill_dev_params(p, &d);

  const size_t P = px * pz;   // the caller's plane stride
  Lev L;
  memset(&L, 0, sizeof(L));
  L.nx = p->nx; L.nz = p->nz; L.px = (int)px; L.pz = (int)pz; L.rw = 0;
  set_spacing(L, p->dx0 / (double)(1 << level), p->dz0 / (double)(1 << level));
  L.P = P;
  L.un = const_cast<double *>(state);
  L.prim = const_cast<double *>(prims);
  L.fx = scratch;
  L.fz = scratch + NCONS * P;
  L.rhsq = rhs_out;                        // the hydro kernels write planes d_t q_D .. d_t q_E here
  L.nfb = reinterpret_cast<unsigned long long *>(scratch + 2 * NCONS * kMaxPlane);
  cudaStream_t s = (cudaStream_t)cuda_stream;
  // every face a divergence reads is written first, so the scratch needs no clearing
  launch_flux_x(L, d, state, p->nx, p->nz, 0.0, 0, 0, s);
  launch_flux_z(L, d, state, p->nx, p->nz, 0.0, 0, 0, s);
  launch_hydro_div(L, d, state, p->nx, p->nz, s);
  if (cudaGetLastError() != cudaSuccess) return SACRA_ERR_CUDA;
  return SACRA_OK;
}
