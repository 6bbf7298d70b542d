// Batched slab marches: many independent Biot instances (own mesh size, time
// order r, permeability field and loads) on one GPU.
//
// Instances that agree in everything but the permeability field and the load
// (mesh, boundary codes, coefficients, r, horizon, slab count, time profiles)
// form a group.  A group of two or more is solved as one batched context
// (biot_setup_batch): its vectors hold all instances level-major, every kernel
// of the slab operator, the preconditioner and the Krylov solver covers all of
// them in one launch, and each Arnoldi step of the whole group is one CUDA graph
// replay.  Groups are processed one after the other by the calling thread.
// Instances that cannot be batched (FP64 solves, groups of one, the 2-D
// manufactured presets whose load depends on the instance's permeability) are
// marched one at a time with a small cache of contexts keyed by shape, swapping
// only the permeability.
#include <algorithm>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <vector>

#include "../../include/biot.h"

namespace {

const double kConstantProfile[4] = {1.0, 0.0, 0.0, 0.0};

bool same_coeffs(const biot_coeffs& a, const biot_coeffs& b) {
  return a.b == b.b && a.invM == b.invM && a.K_dr == b.K_dr && a.lambda == b.lambda && a.mu == b.mu && a.eta == b.eta;
}

bool same_mesh(const biot_mesh& a, const biot_mesh& b) { return std::memcmp(&a, &b, sizeof(biot_mesh)) == 0; }

// loads a batched context can take: the top traction preset (independent of K) or explicit terms
bool batchable(const biot_batch_item& it) {
  if (it.load_kind == BIOT_LOAD_TRACTION_TOP) return true;
  return it.load_kind < 0 && it.nterms >= 0 && it.nterms <= 8 && (it.nterms == 0 || (it.f_terms && it.tcoef));
}

bool same_group(const biot_batch_item& a, const biot_batch_item& b) {
  if (a.r != b.r || a.T != b.T || a.slabs != b.slabs) return false;
  if (!same_mesh(a.mesh, b.mesh) || !same_coeffs(a.coeffs, b.coeffs)) return false;
  if ((a.load_kind >= 0) != (b.load_kind >= 0)) return false;
  if (a.load_kind >= 0) return a.load_kind == b.load_kind;
  if (a.nterms != b.nterms) return false;
  for (int i = 0; i < 4 * a.nterms; ++i)
    if (a.tcoef[i] != b.tcoef[i]) return false;
  return true;
}

int64_t cells_of(const biot_mesh& m) {
  int64_t c = 1;
  for (int d = 0; d < m.dim; ++d) c *= m.n[d];
  return c;
}

// one batched context for the instances idx (all of one group)
void run_group(const biot_batch_item* items, const std::vector<int>& idx, const biot_opts* opts, const biot_solve_opts* sopts,
               cudaStream_t stream, int* st, biot_stats* ss) {
  const int nb = (int)idx.size();
  const biot_batch_item& i0 = items[idx[0]];
  const int64_t nc = cells_of(i0.mesh);
  std::vector<double> K((size_t)nb * nc);
  for (int b = 0; b < nb; ++b) {
    const double* src = items[idx[b]].coeffs.K_cell;
    if (!src) {
      for (int j : idx) st[j] = BIOT_EINVAL;
      return;
    }
    std::memcpy(K.data() + (size_t)b * nc, src, nc * sizeof(double));
  }
  biot_coeffs co = i0.coeffs;
  co.K_cell = K.data();
  biot_t ctx = nullptr;
  int rc = biot_setup_batch(&i0.mesh, &co, i0.r, opts, nb, &ctx);
  if (rc != BIOT_OK) {
    if (std::getenv("BIOT_BATCH_VERBOSE")) std::fprintf(stderr, "biot_solve_batch: group setup failed (%d): %s\n", rc, biot_last_error(nullptr));
    for (int j : idx) st[j] = rc;
    return;
  }
  int64_t n_space = 0;
  biot_sizes(ctx, &n_space, nullptr, nullptr);
  double* fbuf = nullptr;
  std::vector<const double*> terms;
  std::vector<const double*> U0(nb);
  std::vector<double*> Uend(nb);
  int nterms = i0.nterms;
  const double* tco = i0.tcoef;
  if (i0.load_kind >= 0) {
    nterms = 1;
    tco = kConstantProfile;
    if (cudaMalloc((void**)&fbuf, (size_t)nb * n_space * sizeof(double)) != cudaSuccess) rc = BIOT_ENOMEM;
    for (int b = 0; b < nb && rc == BIOT_OK; ++b) {
      rc = biot_load_preset(ctx, i0.load_kind, items[idx[b]].load_value, fbuf + (size_t)b * n_space, stream);
      terms.push_back(fbuf + (size_t)b * n_space);
    }
  } else {
    for (int b = 0; b < nb; ++b)
      for (int m = 0; m < nterms; ++m) terms.push_back(items[idx[b]].f_terms[m]);
  }
  for (int b = 0; b < nb; ++b) {
    U0[b] = items[idx[b]].U0;
    Uend[b] = items[idx[b]].U_end;
  }
  std::vector<int> status(nb, rc);
  std::vector<biot_stats> stats(nb);
  std::memset(stats.data(), 0, stats.size() * sizeof(biot_stats));
  if (rc == BIOT_OK) {
    rc = biot_march_batch(ctx, i0.T, i0.slabs, nterms, terms.data(), tco, U0.data(), Uend.data(), sopts, nullptr, stats.data(),
                          status.data(), stream);
    if (rc != BIOT_OK && std::getenv("BIOT_BATCH_VERBOSE"))
      std::fprintf(stderr, "biot_solve_batch: batched group of %d failed (%d): %s\n", nb, rc, biot_last_error(ctx));
  }
  for (int b = 0; b < nb; ++b) {
    st[idx[b]] = status[b];
    ss[idx[b]] = stats[b];
  }
  if (fbuf) cudaFree(fbuf);
  biot_destroy(ctx);
}

struct Cached {
  biot_mesh mesh;
  biot_coeffs coeffs;  // K_cell ignored in the key
  int r;
  biot_t ctx;
  double* f;  // device buffer for a preset load term
  int64_t n_space;
};

bool same_key(const Cached& c, const biot_batch_item& it) {
  return c.r == it.r && same_mesh(c.mesh, it.mesh) && same_coeffs(c.coeffs, it.coeffs);
}

// one instance at a time, contexts cached by shape (the permeability is swapped)
void run_sequential(const biot_batch_item* items, const std::vector<int>& idx, const biot_opts* opts,
                    const biot_solve_opts* sopts, cudaStream_t stream, int* st, biot_stats* ss) {
  std::vector<Cached> cache;
  for (int i : idx) {
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
      if (cache.size() >= 16) {  // bound the cache
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
        biot_sizes(c.ctx, &c.n_space, nullptr, nullptr);
        cache.push_back(c);
        cc = &cache.back();
      }
    }
    if (rc == BIOT_OK) {
      const double* terms[8];
      const double* tco = it.tcoef;
      int nterms = it.nterms;
      if (it.load_kind >= 0) {
        if (!cc->f && cudaMalloc((void**)&cc->f, cc->n_space * sizeof(double)) != cudaSuccess) rc = BIOT_ENOMEM;
        if (rc == BIOT_OK) rc = biot_load_preset(cc->ctx, it.load_kind, it.load_value, cc->f, stream);
        terms[0] = cc->f;
        nterms = 1;
        tco = kConstantProfile;
      } else {
        for (int m = 0; m < nterms && m < 8; ++m) terms[m] = it.f_terms[m];
      }
      if (rc == BIOT_OK)
        rc = biot_march(cc->ctx, it.T, it.slabs, nterms, terms, tco, it.U0, it.U_end, nullptr, sopts, nullptr, &s, stream);
    }
    if (rc != BIOT_OK && std::getenv("BIOT_BATCH_VERBOSE"))
      std::fprintf(stderr, "biot_solve_batch: instance %d failed (%d): %s\n", i, rc, biot_last_error(cc ? cc->ctx : nullptr));
    st[i] = rc;
    ss[i] = s;
  }
  for (Cached& c : cache) {
    biot_destroy(c.ctx);
    if (c.f) cudaFree(c.f);
  }
}

}  // namespace

extern "C" int biot_solve_batch(const biot_batch_item* items, int count, const biot_opts* opts,
                                const biot_solve_opts* sopts, int workers, int* status, biot_stats* stats) {
  if (!items || count < 0) return BIOT_EINVAL;
  if (count == 0) return BIOT_OK;
  const int cap = workers > 0 ? std::min(workers, 4096) : 64;  // instances per batched context
  const bool mixed = sopts && sopts->mode == BIOT_MIXED;
  std::vector<int> st(count, BIOT_OK);
  std::vector<biot_stats> ss(count);
  std::memset(ss.data(), 0, ss.size() * sizeof(biot_stats));
  cudaStream_t stream = nullptr;
  if (cudaStreamCreateWithFlags(&stream, cudaStreamNonBlocking) != cudaSuccess) return BIOT_ECUDA;
  std::vector<char> taken(count, 0);
  if (mixed) {
    for (int i = 0; i < count; ++i) {
      if (taken[i] || !batchable(items[i])) continue;
      std::vector<int> grp;
      for (int j = i; j < count; ++j)
        if (!taken[j] && batchable(items[j]) && same_group(items[i], items[j])) grp.push_back(j);
      if (grp.size() < 2) continue;
      for (size_t c0 = 0; c0 < grp.size(); c0 += cap) {
        std::vector<int> chunk(grp.begin() + c0, grp.begin() + std::min(grp.size(), c0 + cap));
        for (int j : chunk) taken[j] = 1;
        if (chunk.size() >= 2) run_group(items, chunk, opts, sopts, stream, st.data(), ss.data());
        else taken[chunk[0]] = 0;  // a lone remainder goes the sequential way
      }
    }
  }
  std::vector<int> rest;
  for (int i = 0; i < count; ++i)
    if (!taken[i]) rest.push_back(i);
  run_sequential(items, rest, opts, sopts, stream, st.data(), ss.data());
  cudaStreamDestroy(stream);
  int rc = BIOT_OK;
  for (int i = 0; i < count; ++i) {
    if (status) status[i] = st[i];
    if (stats) stats[i] = ss[i];
    if (st[i] != BIOT_OK && rc == BIOT_OK) rc = st[i];
  }
  return rc;
}
