// Batched slab marches: many independent Biot instances (own mesh size, time
// order r, permeability field and loads) solved concurrently on one GPU.
//
// A host worker pulls instances from a shared counter (one worker for now: see the
// note in biot_solve_batch).  The worker owns a non-blocking CUDA stream and a small
// cache of contexts keyed by
// everything except the permeability (mesh, boundary codes, coefficients, r), so
// instances that share a shape reuse the context's multigrid hierarchy and Krylov
// bases and only swap the cellwise permeability.  The
// GPU interleaves the kernels of all workers' streams; each context's solver runs
// on its own library stream, so instances overlap on the device.  Batch contexts do
// not capture CUDA graphs (a capture on one thread must not overlap the device-wide
// synchronisation that freeing memory implies on another); the concurrent streams
// hide the launch latency instead.
#include <atomic>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <thread>
#include <vector>

#include "../../include/biot.h"

namespace biot {
void ctx_disable_graphs(biot_t c);
}

namespace {

struct Cached {
  biot_mesh mesh;
  biot_coeffs coeffs;  // K_cell ignored in the key
  int r;
  biot_t ctx;
  double* f;  // device buffer for a preset load term
  int64_t n_space;
};

bool same_key(const Cached& c, const biot_batch_item& it) {
  if (c.r != it.r) return false;
  if (std::memcmp(&c.mesh, &it.mesh, sizeof(biot_mesh)) != 0) return false;
  const biot_coeffs& a = c.coeffs;
  const biot_coeffs& b = it.coeffs;
  return a.b == b.b && a.invM == b.invM && a.K_dr == b.K_dr && a.lambda == b.lambda && a.mu == b.mu && a.eta == b.eta;
}

}  // namespace

extern "C" int biot_solve_batch(const biot_batch_item* items, int count, const biot_opts* opts,
                                const biot_solve_opts* sopts, int workers, int* status, biot_stats* stats) {
  if (!items || count < 0) return BIOT_EINVAL;
  if (count == 0) return BIOT_OK;
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return BIOT_ECUDA;
  // Several concurrent workers raised an illegal-address fault on the GB300 (after the
  // first round of instances; not with blocking launches); until its cause is found the
  // instances run on one worker, in order, with the context cache.
  (void)workers;
  workers = 1;
  std::atomic<int> next{0};
  std::vector<int> st(count, BIOT_OK);
  std::vector<biot_stats> ss(count);
  auto work = [&]() {
    cudaSetDevice(dev);
    cudaStream_t stream = nullptr;
    if (cudaStreamCreateWithFlags(&stream, cudaStreamNonBlocking) != cudaSuccess) {
      for (int i; (i = next.fetch_add(1)) < count;) st[i] = BIOT_ECUDA;
      return;
    }
    std::vector<Cached> cache;
    for (int i; (i = next.fetch_add(1)) < count;) {
      const biot_batch_item& it = items[i];
      biot_stats s;
      std::memset(&s, 0, sizeof(s));
      int rc = BIOT_OK;
      Cached* cc = nullptr;
      for (Cached& c : cache)
        if (same_key(c, it)) { cc = &c; break; }
      if (cc) {
        rc = biot_set_permeability(cc->ctx, it.coeffs.K_cell);
      } else {
        if (cache.size() >= 16) {  // bound the per-worker cache
          biot_destroy(cache.front().ctx);
          if (cache.front().f) cudaFree(cache.front().f);
          cache.erase(cache.begin());
        }
        Cached c;
        std::memset(&c, 0, sizeof(c));
        c.mesh = it.mesh;
        c.coeffs = it.coeffs;
        c.r = it.r;
        rc = biot_setup(&it.mesh, &it.coeffs, it.r, opts, &c.ctx);
        if (rc == BIOT_OK) {
          biot::ctx_disable_graphs(c.ctx);
          biot_sizes(c.ctx, &c.n_space, nullptr, nullptr);
          cache.push_back(c);
          cc = &cache.back();
        }
      }
      if (rc == BIOT_OK) {
        const double* terms[8];
        const double* tco = it.tcoef;
        static const double constant_profile[4] = {1.0, 0.0, 0.0, 0.0};
        int nterms = it.nterms;
        if (it.load_kind >= 0) {
          if (!cc->f && cudaMalloc((void**)&cc->f, cc->n_space * sizeof(double)) != cudaSuccess) rc = BIOT_ENOMEM;
          if (rc == BIOT_OK) rc = biot_load_preset(cc->ctx, it.load_kind, it.load_value, cc->f, stream);
          terms[0] = cc->f;
          nterms = 1;
          tco = constant_profile;
        } else {
          for (int m = 0; m < nterms && m < 8; ++m) terms[m] = it.f_terms[m];
        }
        if (rc == BIOT_OK)
          rc = biot_march(cc->ctx, it.T, it.slabs, nterms, terms, tco, it.U0, it.U_end, nullptr, sopts, nullptr, &s, stream);
      }
      if (rc != BIOT_OK && std::getenv("BIOT_BATCH_VERBOSE"))
        std::fprintf(stderr, "biot_solve_batch: instance %d failed (%d): %s\n", i, rc,
                     biot_last_error(cc ? cc->ctx : nullptr));
      st[i] = rc;
      ss[i] = s;
    }
    for (Cached& c : cache) {
      biot_destroy(c.ctx);
      if (c.f) cudaFree(c.f);
    }
    cudaStreamDestroy(stream);
  };
  std::vector<std::thread> pool;
  for (int w = 0; w < workers; ++w) pool.emplace_back(work);
  for (std::thread& t : pool) t.join();
  int rc = BIOT_OK;
  for (int i = 0; i < count; ++i) {
    if (status) status[i] = st[i];
    if (stats) stats[i] = ss[i];
    if (st[i] != BIOT_OK && rc == BIOT_OK) rc = st[i];
  }
  return rc;
}
