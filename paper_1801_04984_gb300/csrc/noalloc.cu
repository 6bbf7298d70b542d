// Allocation-free variant of the flux-pressure Schur complement apply.
//
// Some callers cannot call cudaMalloc at the point where they need this
// operator: applications whose caching allocator has already reserved the whole
// device, latency-critical loops where cudaMalloc's implicit device-wide
// synchronisation is not acceptable, and embedded or real-time hosts that forbid
// dynamic device allocation after start-up.  This entry point therefore keeps its
// flux-grid scratch vector in a file-scope __device__ array instead of the
// context's lazily allocated workspace.  The paper has no counterpart: this is an
// interface convenience around the preconditioner piece of §Monolithic Approach.
#include <cstring>
#include <mutex>

#include "../../include/biot.h"
#include "internal.h"

namespace {

// Scratch for one flux-grid vector.  Every GPU that loads the library holds it
// until the process exits.  Every call shares it and overwrites it completely.
constexpr long long kNoAllocMaxFlux = 1LL << 20;  // flux DoFs (8 MiB of FP64)
static __device__ __align__(256) double g_noalloc_flux[kNoAllocMaxFlux];

constexpr int kMaxDevices = 64;
std::mutex g_mu;
double* g_addr[kMaxDevices] = {nullptr};

}  // namespace

// Defined in api.cu: grid, tables and per-cell data of a context (no allocation).
namespace biot {
struct CtxView {
  const Grid* g;
  const TabT<double>* t64;
  const double* dmq64;
  double invM, beta;
  int nb;
  int lumped_flux;
};
bool ctx_view(biot_t ctx, CtxView* v);
void ctx_set_error(biot_t ctx, const char* msg);
}  // namespace biot

extern "C" int biot_schur_apply_noalloc(biot_t ctx, double tau, const double* in, double* out, void* stream) {
  using namespace biot;
  CtxView v;
  if (!ctx_view(ctx, &v)) return BIOT_EINVAL;
  if (v.nb != 1) {
    ctx_set_error(ctx, "schur_apply_noalloc: batched contexts (biot_setup_batch) are not supported; use a context of biot_setup");
    return BIOT_EINVAL;
  }
  if (!v.lumped_flux) {
    ctx_set_error(ctx, "schur_apply_noalloc: the context inverts the Darcy mass exactly (flux_mass_exact = 1); this entry "
                       "point applies only the lumped-Darcy-mass Schur complement");
    return BIOT_EINVAL;
  }
  if (!in || !out || !(tau > 0)) {
    ctx_set_error(ctx, "schur_apply_noalloc: NULL vector or tau <= 0");
    return BIOT_EINVAL;
  }
  const Grid& g = *v.g;
  const long long nq = g.nq[0] + g.nq[1] + g.nq[2];
  if (nq > kNoAllocMaxFlux) {
    ctx_set_error(ctx, "schur_apply_noalloc: the mesh has more flux DoFs than the static scratch holds (1048576)");
    return BIOT_EINVAL;
  }
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) {
    ctx_set_error(ctx, "schur_apply_noalloc: no usable current CUDA device");
    return BIOT_ECUDA;
  }
  double* scratch = nullptr;
  {
    // set-up once per device, with that device current: the symbol's host-side
    // name is only a stand-in, its device address has to be queried
    std::lock_guard<std::mutex> lk(g_mu);
    if (!g_addr[dev]) {
      void* p = nullptr;
      cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_flux);
      if (e != cudaSuccess) {
        ctx_set_error(ctx, cudaGetErrorString(e));
        return BIOT_ECUDA;
      }
      g_addr[dev] = static_cast<double*>(p);
    }
    scratch = g_addr[dev];
  }
  cudaStream_t st = (cudaStream_t)stream;
  if (cudaMemsetAsync(out, 0, g.N * sizeof(double), st) != cudaSuccess) {
    ctx_set_error(ctx, "schur_apply_noalloc: cudaMemsetAsync failed");
    return BIOT_ECUDA;
  }
  double cm[1] = {v.invM + v.beta};
  launch_schur_apply<double>(g, *v.t64, in + g.offp, g.Np, v.dmq64, scratch, nq, tau, cm, out + g.offp, g.Np, 1, st);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) {
    ctx_set_error(ctx, cudaGetErrorString(e));
    return BIOT_ECUDA;
  }
  return BIOT_OK;
}
