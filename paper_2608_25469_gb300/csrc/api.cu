// C ABI of the library (include/hsma.h): argument checks, quick returns, the
// dispatcher of Section 4.1 and the block-size lookup of Section 4.3.2.
#include <cuda_runtime.h>

#include <algorithm>
#include <atomic>
#include <cmath>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <mutex>
#include <string>
#include <vector>

#include "../../include/hsma.h"
#include "blocked.h"
#include "common.cuh"
#include "gen.h"
#include "mixed.h"
#include "small.h"
#include "trace.h"
#include "workspace.h"

namespace {

bool valid_dtype(int d) { return d >= HSMA_R64 && d <= HSMA_C64; }

// Column-packed varlen batch unless HSMA_VB_PACKED=0 (read once).
bool packed_enabled() {
  static const bool on = [] {
    const char *e = std::getenv("HSMA_VB_PACKED");
    return !(e != nullptr && std::atoi(e) == 0);
  }();
  return on;
}
bool is_complex(int d) { return d == HSMA_C128 || d == HSMA_C64; }
bool valid_diag(int d) { return d == HSMA_NON_UNIT || d == HSMA_UNIT; }

// ---------------------------------------------------------------------------
// Block-size table (Section 4.3.2): offline profiling keeps the best N_B per
// (dtype, scale); at run time the nearest profiled scale wins.  Distance is
// measured in (log m, log n).  Entries come from the autotuner's sweep on this
// GPU (tuning/gb300.txt); hsma_tuning_load replaces them.
// ---------------------------------------------------------------------------
struct TuneEntry {
  int dtype;
  int64_t m, n;
  int nb;
  int tile = 0;                     // HSMA_TILE_*, 0 = by n
  int split_k = HSMA_SPLITK_AUTO;
  int looking = HSMA_LOOK_RIGHT;
  int panel_cols = kEmuPanelColsDefault;  // emulated products
};

#include "tuning_table.inc"

std::mutex g_tune_mu;
std::vector<TuneEntry> g_tune;  // empty = compiled table

TuneEntry lookup(int dtype, int64_t m, int64_t n) {
  std::lock_guard<std::mutex> lk(g_tune_mu);
  const TuneEntry *tab = g_tune.empty() ? kCompiledTable : g_tune.data();
  const size_t cnt = g_tune.empty() ? sizeof(kCompiledTable) / sizeof(kCompiledTable[0]) : g_tune.size();
  // R64_IR and R32 tune as R32_BF16 (their blocked solves run that path), C64 as C128;
  // fall back to R64 entries if a dtype has none (emulated-products keys to their defaults)
  const bool emu_key = dtype == kEmulatedTableDtype(HSMA_R64) || dtype == kEmulatedTableDtype(HSMA_C128);
  const int want = (dtype == HSMA_R64_IR || dtype == HSMA_R32) ? HSMA_R32_BF16
                   : dtype == HSMA_C64                         ? HSMA_C128
                                                               : dtype;
  for (int pass = 0; pass < (emu_key ? 1 : 2); ++pass) {
    const int d = pass == 0 ? want : HSMA_R64;
    double best = 1e300;
    const TuneEntry *pick = nullptr;
    for (size_t k = 0; k < cnt; ++k) {
      if (tab[k].dtype != d) continue;
      const double dm = std::log((double)std::max<int64_t>(m, 1)) - std::log((double)tab[k].m);
      const double dn = std::log((double)std::max<int64_t>(n, 1)) - std::log((double)tab[k].n);
      const double dist = dm * dm + dn * dn;
      if (dist < best) {
        best = dist;
        pick = &tab[k];
      }
    }
    if (pick != nullptr) return *pick;
  }
  TuneEntry e{dtype, m, n, emu_key ? kHsmaEmulatedNb : 128};
  return e;
}

bool valid_table_dtype(int d) {
  return valid_dtype(d) || d == kEmulatedTableDtype(HSMA_R64) || d == kEmulatedTableDtype(HSMA_C128);
}

bool valid_tile(int t) { return t >= 0 && t <= HSMA_TILE_128x8; }
bool valid_split(int v) { return v >= 0 && v <= HSMA_SPLITK_OFF; }
bool valid_look(int v) { return v >= 0 && v <= HSMA_LOOK_LEFT; }
bool valid_panel(int v) { return v == 0 || (v >= 512 && v <= 8192 && v % 64 == 0); }

hsma_status_t make_plan(int dtype, int64_t m, int64_t n, const hsma_opts_t *opts, hsma_plan_t *p) {
  std::memset(p, 0, sizeof(*p));
  int path = opts ? opts->path : HSMA_PATH_AUTO;
  if (path < HSMA_PATH_AUTO || path > HSMA_PATH_BLOCKED) return HSMA_ERR_INVALID_ARG;
  if (opts && (opts->fp64_products < 0 || opts->fp64_products > 1)) return HSMA_ERR_INVALID_ARG;
  const bool small_ok = m <= 64 && hsma_small_dtype(dtype);
  if (path == HSMA_PATH_AUTO) path = small_ok ? HSMA_PATH_SMALL : HSMA_PATH_BLOCKED;
  if (path == HSMA_PATH_SMALL && !small_ok) return HSMA_ERR_UNSUPPORTED;
  p->path = path;
  if (path == HSMA_PATH_SMALL) {
    const bool cplx_ = is_complex(dtype);
    int g = opts ? opts->groups : 0;
    if (g != 0) {
      if (g != 1 && g != 2 && g != 4 && g != 8 && g != 16 && g != 32) return HSMA_ERR_INVALID_ARG;
      if (!hsma_small_g_ok(g, (int)m, cplx_)) return HSMA_ERR_INVALID_ARG;
    } else {
      g = hsma_small_pick_g_single((int)std::max<int64_t>(m, 1), (int)std::min<int64_t>(n, 1 << 30), cplx_,
                                   hsma_sm_count());
    }
    p->groups = g;
  } else {
    int nb = opts ? opts->nb : 0;
    if (nb != 0 && (nb < 16 || nb > 512 || nb % 16 != 0)) return HSMA_ERR_INVALID_ARG;
    if (opts && (!valid_tile(opts->tile) || !valid_split(opts->split_k) || !valid_look(opts->looking) ||
                 !valid_panel(opts->panel_cols)))
      return HSMA_ERR_INVALID_ARG;
    // the table's entry for this scale (the emulated-products entries when the
    // FP64 products are emulated: the option, or complex64's widened solve);
    // every option the caller gives overrides its field
    const bool emu = dtype == HSMA_C64 || ((dtype == HSMA_R64 || dtype == HSMA_C128) && opts && opts->fp64_products == 1);
    const TuneEntry e = lookup(emu ? kEmulatedTableDtype(dtype == HSMA_C64 ? HSMA_C128 : dtype) : dtype, m, n);
    p->nb = nb != 0 ? nb : e.nb;
    p->tile = opts && opts->tile ? opts->tile : e.tile;
    p->split_k = opts && opts->split_k ? opts->split_k : e.split_k;
    p->looking = opts && opts->looking ? opts->looking : e.looking;
    p->panel_cols = opts && opts->panel_cols ? opts->panel_cols : e.panel_cols;
  }
  return HSMA_OK;
}

size_t elem_bytes(int dtype) {
  switch (dtype) {
    case HSMA_C128: return 16;
    case HSMA_R32_BF16:
    case HSMA_R32: return 4;
    default: return 8;
  }
}

bool alpha_is_zero(int dtype, const void *alpha) {
  const double *a = static_cast<const double *>(alpha);
  if (is_complex(dtype)) return a[0] == 0.0 && a[1] == 0.0;
  return a[0] == 0.0;
}

}  // namespace

extern "C" {

}  // extern "C"

hsma_status_t hsma_make_plan(int dtype, int64_t m, int64_t n, const hsma_opts_t *opts, hsma_plan_t *out) {
  return make_plan(dtype, m, n, opts, out);
}

extern "C" {

const char *hsma_status_string(int s) {
  switch (s) {
    case HSMA_OK: return "HSMA_OK";
    case HSMA_ERR_INVALID_ARG: return "HSMA_ERR_INVALID_ARG";
    case HSMA_ERR_UNSUPPORTED: return "HSMA_ERR_UNSUPPORTED";
    case HSMA_ERR_NO_MEMORY: return "HSMA_ERR_NO_MEMORY";
    case HSMA_ERR_CUDA: return "HSMA_ERR_CUDA";
    case HSMA_ERR_TIMEOUT: return "HSMA_ERR_TIMEOUT";
    case HSMA_ERR_NOT_CONVERGED: return "HSMA_ERR_NOT_CONVERGED";
    case HSMA_ERR_BUSY: return "HSMA_ERR_BUSY";
    default: return "HSMA_ERR_UNKNOWN";
  }
}

const char *hsma_version(void) { return "0.1.0"; }

hsma_status_t hsma_plan(int dtype, int64_t m, int64_t n, hsma_plan_t *out) {
  if (!valid_dtype(dtype) || m < 0 || n < 0 || out == nullptr) return HSMA_ERR_INVALID_ARG;
  return make_plan(dtype, m, n, nullptr, out);
}

double hsma_small_cost(int dtype, int64_t m, int64_t n, int32_t groups) {
  if (m < 1 || m > 64 || n < 0 || !hsma_small_dtype(dtype)) return -1.0;
  if (groups != 1 && groups != 2 && groups != 4 && groups != 8 && groups != 16 && groups != 32) return -1.0;
  if (!hsma_small_g_ok(groups, (int)m, is_complex(dtype))) return -1.0;
  return hsma_small_total_instr((int)m, (int)n, groups, is_complex(dtype));
}

hsma_status_t hsma_tuning_load(const char *path) {
  std::lock_guard<std::mutex> lk(g_tune_mu);
  if (path == nullptr) {
    g_tune.clear();
    return HSMA_OK;
  }
  FILE *f = std::fopen(path, "r");
  if (!f) return HSMA_ERR_INVALID_ARG;
  std::vector<TuneEntry> t;
  char line[256];
  while (std::fgets(line, sizeof line, f)) {
    if (line[0] == '#' || line[0] == '\n') continue;
    int d, nb, tile = 0, split = HSMA_SPLITK_AUTO, look = HSMA_LOOK_RIGHT, panel = kEmuPanelColsDefault;
    long long m, n;
    const int got = std::sscanf(line, "%d %lld %lld %d %d %d %d %d", &d, &m, &n, &nb, &tile, &split, &look, &panel);
    if ((got != 4 && got != 8) || !valid_table_dtype(d) || m < 1 || n < 1 || nb < 16 || nb > 512 || nb % 16 != 0 ||
        !valid_tile(tile) || split < 1 || split > 2 || look < 1 || look > 2 || panel == 0 || !valid_panel(panel)) {
      std::fclose(f);
      return HSMA_ERR_INVALID_ARG;
    }
    t.push_back(TuneEntry{d, m, n, nb, tile, split, look, panel});
  }
  std::fclose(f);
  if (t.empty()) return HSMA_ERR_INVALID_ARG;
  g_tune.swap(t);
  return HSMA_OK;
}

hsma_status_t hsma_trsm_llnn_ex(int dtype, int diag, int64_t m, int64_t n, const void *alpha, const void *A,
                                int64_t lda, void *B, int64_t ldb, void *stream, const hsma_opts_t *opts,
                                hsma_info_t *info) {
  if (!valid_dtype(dtype) || !valid_diag(diag)) return HSMA_ERR_INVALID_ARG;
  if (m < 0 || n < 0) return HSMA_ERR_INVALID_ARG;
  const int64_t lo = std::max<int64_t>(1, m);
  if (lda < lo || ldb < lo) return HSMA_ERR_INVALID_ARG;
  if (m > INT32_MAX || n > INT32_MAX) return HSMA_ERR_UNSUPPORTED;
  if (info) std::memset(info, 0, sizeof(*info));
  if (m == 0 || n == 0) return HSMA_OK;
  if (alpha == nullptr || A == nullptr || B == nullptr) return HSMA_ERR_INVALID_ARG;
  hsma_plan_t plan;
  hsma_status_t s = make_plan(dtype, m, n, opts, &plan);
  if (s != HSMA_OK) return s;
  if (info) info->plan = plan;
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  if (alpha_is_zero(dtype, alpha)) {
    const size_t eb = elem_bytes(dtype);
    HSMA_CUDA_TRY(cudaMemset2DAsync(B, (size_t)ldb * eb, 0, (size_t)m * eb, (size_t)n, st));
    return HSMA_OK;
  }
  const int unit = diag == HSMA_UNIT;
  const double *al = static_cast<const double *>(alpha);
  switch (dtype) {
    case HSMA_R64:
    case HSMA_C128:
      if (plan.path == HSMA_PATH_SMALL)
        return hsma_small_single(dtype, plan.groups, A, lda, B, ldb, (int)m, (int)n, al, unit, st);
      if (opts != nullptr && opts->fp64_products == 1)
        return hsma_blocked_emulated(dtype, plan.nb, plan.panel_cols, A, lda, B, ldb, m, n, al, unit, st);
      {
        HsmaBlockedCfg cfg;
        cfg.nb = plan.nb;
        cfg.tile = plan.tile;
        cfg.split_k = plan.split_k;
        cfg.looking = plan.looking;
        return hsma_blocked_solve(dtype, cfg, A, lda, B, ldb, m, n, al, unit, st);
      }
    case HSMA_R32_BF16:
      return hsma_mixed_r32(plan.nb, opts ? opts->bf16_terms : 0, static_cast<const float *>(A), lda,
                            static_cast<float *>(B), ldb, m, n, al[0], unit, st);
    case HSMA_R64_IR:
      return hsma_mixed_ir(plan.nb, opts, static_cast<const double *>(A), lda, static_cast<double *>(B), ldb, m,
                           n, al[0], unit, st, info);
    case HSMA_R32:
      if (plan.path == HSMA_PATH_SMALL)
        return hsma_small_single(dtype, plan.groups, A, lda, B, ldb, (int)m, (int)n, al, unit, st);
      return hsma_mixed_r32(plan.nb, opts ? opts->bf16_terms : 0, static_cast<const float *>(A), lda,
                            static_cast<float *>(B), ldb, m, n, al[0], unit, st);
    case HSMA_C64:
      if (plan.path == HSMA_PATH_SMALL)
        return hsma_small_single(dtype, plan.groups, A, lda, B, ldb, (int)m, (int)n, al, unit, st);
      return hsma_c64_blocked(plan.nb, plan.panel_cols, A, lda, B, ldb, m, n, al, unit, st);
    default:
      return HSMA_ERR_INVALID_ARG;
  }
}

hsma_status_t hsma_trsm_llnn(int dtype, int diag, int64_t m, int64_t n, const void *alpha, const void *A,
                             int64_t lda, void *B, int64_t ldb, void *stream) {
  return hsma_trsm_llnn_ex(dtype, diag, m, n, alpha, A, lda, B, ldb, stream, nullptr, nullptr);
}

hsma_status_t hsma_trsm_llnn_vbatched(int dtype, int diag, int32_t batch, const int32_t *d_m, const int32_t *d_n,
                                      const void *alpha, const void *const *d_A, const int32_t *d_lda,
                                      void *const *d_B, const int32_t *d_ldb, int32_t max_m, int32_t max_n,
                                      uint32_t *d_status, void *stream) {
  return hsma_trsm_vbatched(dtype, HSMA_LEFT, HSMA_LOWER, HSMA_NO_TRANS, diag, batch, d_m, d_n, alpha, d_A, d_lda,
                            d_B, d_ldb, max_m, max_n, d_status, stream);
}

}  // extern "C"

namespace {

__global__ void or_status_kernel(uint32_t *status, uint32_t bits) { atomicOr(status, bits); }

// A batch whose host bound max_m exceeds 64, read back to the host: the sizes,
// pointers and (factor solves) pivot pointers of every instance.  The stream
// is waited for once.
struct HostBatch {
  std::vector<int32_t> m, n, lda, ldb;
  std::vector<const void *> A;
  std::vector<void *> B;
  std::vector<const int32_t *> piv;
};

hsma_status_t read_batch(int32_t batch, const int32_t *d_m, const int32_t *d_n, const int32_t *d_lda,
                         const int32_t *d_ldb, const void *const *d_A, void *const *d_B,
                         const int32_t *const *d_ipiv, cudaStream_t st, HostBatch &h) {
  const size_t b = (size_t)batch;
  h.m.resize(b);
  h.n.resize(b);
  h.lda.resize(b);
  h.ldb.resize(b);
  h.A.resize(b);
  h.B.resize(b);
  h.piv.assign(b, nullptr);
  HSMA_CUDA_TRY(cudaMemcpyAsync(h.m.data(), d_m, 4 * b, cudaMemcpyDeviceToHost, st));
  HSMA_CUDA_TRY(cudaMemcpyAsync(h.n.data(), d_n, 4 * b, cudaMemcpyDeviceToHost, st));
  HSMA_CUDA_TRY(cudaMemcpyAsync(h.lda.data(), d_lda, 4 * b, cudaMemcpyDeviceToHost, st));
  HSMA_CUDA_TRY(cudaMemcpyAsync(h.ldb.data(), d_ldb, 4 * b, cudaMemcpyDeviceToHost, st));
  HSMA_CUDA_TRY(cudaMemcpyAsync(h.A.data(), d_A, sizeof(void *) * b, cudaMemcpyDeviceToHost, st));
  HSMA_CUDA_TRY(cudaMemcpyAsync(h.B.data(), d_B, sizeof(void *) * b, cudaMemcpyDeviceToHost, st));
  if (d_ipiv != nullptr)
    HSMA_CUDA_TRY(cudaMemcpyAsync(h.piv.data(), d_ipiv, sizeof(void *) * b, cudaMemcpyDeviceToHost, st));
  HSMA_CUDA_TRY(cudaStreamSynchronize(st));
  return HSMA_OK;
}

// Every instance with m > 64 through `solve1(b)` on the stream; invalid ones
// (n < 0, ld < m, null pointer) are skipped and their HSMA_DEVERR_* bits ORed
// into d_status.
template <class F>
hsma_status_t solve_large(const HostBatch &h, uint32_t *d_status, cudaStream_t st, F solve1) {
  uint32_t bad = 0;
  hsma_status_t s = HSMA_OK;
  for (size_t b = 0; b < h.m.size() && s == HSMA_OK; ++b) {
    const int32_t m = h.m[b];
    if (m <= 64) continue;
    if (h.n[b] < 0 || h.lda[b] < m || h.ldb[b] < m) {
      bad |= HSMA_DEVERR_BAD_SIZE;
      continue;
    }
    if (h.n[b] == 0) continue;
    if (h.A[b] == nullptr || h.B[b] == nullptr) {
      bad |= HSMA_DEVERR_NULL_PTR;
      continue;
    }
    s = solve1(b);
  }
  if (s == HSMA_OK && bad != 0 && d_status != nullptr) {
    or_status_kernel<<<1, 1, 0, st>>>(d_status, bad);
    hsma_count_launches(1);
    s = hsma_from_cuda(cudaGetLastError());
  }
  return s;
}

}  // namespace

extern "C" {

hsma_status_t hsma_trsm_vbatched(int dtype, int side, int uplo, int trans, int diag, int32_t batch,
                                 const int32_t *d_m, const int32_t *d_n, const void *alpha, const void *const *d_A,
                                 const int32_t *d_lda, void *const *d_B, const int32_t *d_ldb, int32_t max_m,
                                 int32_t max_n, uint32_t *d_status, void *stream) {
  if (!hsma_small_dtype(dtype)) {
    return valid_dtype(dtype) ? HSMA_ERR_UNSUPPORTED : HSMA_ERR_INVALID_ARG;
  }
  if ((side != HSMA_LEFT && side != HSMA_RIGHT) || (uplo != HSMA_LOWER && uplo != HSMA_UPPER) ||
      trans < HSMA_NO_TRANS || trans > HSMA_CONJ_TRANS)
    return HSMA_ERR_INVALID_ARG;
  if (side == HSMA_RIGHT) return HSMA_ERR_UNSUPPORTED;
  if (!valid_diag(diag) || batch < 0 || max_m < 0 || max_n < 0) return HSMA_ERR_INVALID_ARG;
  if (batch > (1 << 24) - 1) return HSMA_ERR_UNSUPPORTED;
  if (batch == 0) return HSMA_OK;
  if (alpha == nullptr || d_m == nullptr || d_n == nullptr || d_A == nullptr || d_lda == nullptr ||
      d_B == nullptr || d_ldb == nullptr)
    return HSMA_ERR_INVALID_ARG;
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  const bool large = max_m > 64;
  HostBatch hb;
  if (large) {
    hsma_status_t r = read_batch(batch, d_m, d_n, d_lda, d_ldb, d_A, d_B, nullptr, st, hb);
    if (r != HSMA_OK) return r;
  }
  void *scratch = nullptr;
  // complex128 runs the column-packed batch for every left-side variant (the
  // FP64 pipe binds, so full warp tiles pay; the variants through the index
  // map), the other dtypes the per-instance kernel (with the same map)
  const bool packed = hsma_vbatched_packed_dtype(dtype) && packed_enabled();
  hsma_status_t s = hsma_ws_alloc(
      &scratch, packed ? hsma_vbatched_packed_scratch_bytes(dtype, batch, max_m) : hsma_vbatched_scratch_bytes(batch),
      st);
  if (s != HSMA_OK) return s;
  if (packed)
    s = hsma_small_vbatched_packed(dtype, batch, max_m, d_m, d_n, static_cast<const double *>(alpha), d_A, d_lda,
                                   d_B, d_ldb, diag == HSMA_UNIT, d_status, scratch, st, 0, uplo, trans);
  else
    s = hsma_small_vbatched(dtype, batch, d_m, d_n, static_cast<const double *>(alpha), d_A, d_lda, d_B, d_ldb,
                            diag == HSMA_UNIT, d_status, static_cast<int32_t *>(scratch), st, uplo, trans,
                            large ? 1 : 0);
  hsma_status_t f = hsma_ws_free(scratch, st);
  if (s == HSMA_OK && f == HSMA_OK && large)
    s = solve_large(hb, d_status, st, [&](size_t b) {
      return hsma_trsm(dtype, HSMA_LEFT, uplo, trans, diag, hb.m[b], hb.n[b], alpha, hb.A[b], hb.lda[b], hb.B[b],
                       hb.ldb[b], stream, nullptr, nullptr);
    });
  return s != HSMA_OK ? s : f;
}

static hsma_status_t factor_solve_vbatched(int dtype, int32_t batch, const int32_t *d_m, const int32_t *d_n,
                                           const void *alpha, const void *const *d_LU, const int32_t *d_lda,
                                           const int32_t *const *d_ipiv, void *const *d_B, const int32_t *d_ldb,
                                           int32_t max_m, int32_t max_n, uint32_t *d_status, void *stream,
                                           int chol) {
  if (!hsma_small_dtype(dtype)) {
    return valid_dtype(dtype) ? HSMA_ERR_UNSUPPORTED : HSMA_ERR_INVALID_ARG;
  }
  if (batch < 0 || max_m < 0 || max_n < 0) return HSMA_ERR_INVALID_ARG;
  if (batch > (1 << 24) - 1) return HSMA_ERR_UNSUPPORTED;
  if (batch == 0) return HSMA_OK;
  if (alpha == nullptr || d_m == nullptr || d_n == nullptr || d_LU == nullptr || d_lda == nullptr ||
      d_B == nullptr || d_ldb == nullptr)
    return HSMA_ERR_INVALID_ARG;
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  const bool large = max_m > 64;
  HostBatch hb;
  if (large) {
    hsma_status_t r = read_batch(batch, d_m, d_n, d_lda, d_ldb, d_LU, d_B, chol ? nullptr : d_ipiv, st, hb);
    if (r != HSMA_OK) return r;
  }
  void *scratch = nullptr;
  hsma_status_t s, f;
  if (hsma_vbatched_packed_dtype(dtype) && packed_enabled()) {
    // The row interchanges as their own pass, then the two triangular solves
    // as separate launches of the column-packed batch: the lower factor (the
    // paper's case), then the second factor through the index map (U, or
    // L^H).  The same arithmetic as the fused kernel, bit for bit; faster,
    // since the fused kernel cannot use the packed batch.
    auto al = [](size_t v) { return (v + 255) & ~(size_t)255; };
    const bool piv = !chol && d_ipiv != nullptr;
    const size_t me_b = piv ? al(sizeof(int32_t) * (size_t)batch) : 0;
    const size_t pk_b = al(hsma_vbatched_packed_scratch_bytes(dtype, batch, max_m));
    s = hsma_ws_alloc(&scratch, me_b + pk_b, st);
    if (s != HSMA_OK) return s;
    unsigned char *q = static_cast<unsigned char *>(scratch);
    int32_t *m_eff = reinterpret_cast<int32_t *>(q);
    const int32_t *ms = piv ? m_eff : d_m;
    const double *al2 = static_cast<const double *>(alpha);
    const bool azero = al2[0] == 0.0 && al2[1] == 0.0;
    const double one[2] = {1.0, 0.0};
    if (piv)
      s = hsma_small_lu_pivots(dtype, batch, d_m, d_n, d_lda, d_ldb, d_LU, d_B, d_ipiv, m_eff, d_status, st);
    if (s == HSMA_OK)
      s = hsma_small_vbatched_packed(dtype, batch, max_m, ms, d_n, al2, d_LU, d_lda, d_B, d_ldb, chol ? 0 : 1,
                                     d_status, q + me_b, st);
    if (s == HSMA_OK && !azero)  // alpha = 0: X = 0 without reading the factors
      s = hsma_small_vbatched_packed(dtype, batch, max_m, ms, d_n, one, d_LU, d_lda, d_B, d_ldb, 0, d_status,
                                     q + me_b, st, 0, chol ? HSMA_LOWER : HSMA_UPPER,
                                     chol ? HSMA_CONJ_TRANS : HSMA_NO_TRANS);
  } else {
    s = hsma_ws_alloc(&scratch, hsma_vbatched_scratch_bytes(batch), st);
    if (s != HSMA_OK) return s;
    s = hsma_small_getrs_vbatched(dtype, batch, d_m, d_n, static_cast<const double *>(alpha), d_LU, d_lda, d_ipiv,
                                  d_B, d_ldb, d_status, static_cast<int32_t *>(scratch), st, chol, large ? 1 : 0);
  }
  f = hsma_ws_free(scratch, st);
  if (s == HSMA_OK && f == HSMA_OK && large)
    s = solve_large(hb, d_status, st, [&](size_t b) {
      return chol ? hsma_potrs(dtype, hb.m[b], hb.n[b], alpha, hb.A[b], hb.lda[b], hb.B[b], hb.ldb[b], stream,
                               nullptr)
                  : hsma_getrs(dtype, hb.m[b], hb.n[b], alpha, hb.A[b], hb.lda[b], hb.piv[b], hb.B[b], hb.ldb[b],
                               stream, nullptr);
    });
  return s != HSMA_OK ? s : f;
}

hsma_status_t hsma_getrs_vbatched(int dtype, int32_t batch, const int32_t *d_m, const int32_t *d_n,
                                  const void *alpha, const void *const *d_LU, const int32_t *d_lda,
                                  const int32_t *const *d_ipiv, void *const *d_B, const int32_t *d_ldb,
                                  int32_t max_m, int32_t max_n, uint32_t *d_status, void *stream) {
  return factor_solve_vbatched(dtype, batch, d_m, d_n, alpha, d_LU, d_lda, d_ipiv, d_B, d_ldb, max_m, max_n,
                               d_status, stream, 0);
}

hsma_status_t hsma_potrs_vbatched(int dtype, int32_t batch, const int32_t *d_m, const int32_t *d_n,
                                  const void *alpha, const void *const *d_L, const int32_t *d_lda, void *const *d_B,
                                  const int32_t *d_ldb, int32_t max_m, int32_t max_n, uint32_t *d_status,
                                  void *stream) {
  return factor_solve_vbatched(dtype, batch, d_m, d_n, alpha, d_L, d_lda, nullptr, d_B, d_ldb, max_m, max_n,
                               d_status, stream, 1);
}

hsma_status_t hsma_gen_matrix(int dtype, int kind, uint64_t seed, int64_t inst, int64_t m, int64_t cols, void *dst,
                              int64_t ld, void *stream) {
  if ((dtype != HSMA_R64 && dtype != HSMA_C128) || kind < 0 || kind > 2) return HSMA_ERR_INVALID_ARG;
  if (m < 0 || cols < 0 || ld < std::max<int64_t>(1, m) || inst < -1) return HSMA_ERR_INVALID_ARG;
  if (kind != 1 && cols != m) return HSMA_ERR_INVALID_ARG;
  if (m * cols > 0 && dst == nullptr) return HSMA_ERR_INVALID_ARG;
  return hsma_gen_launch(dtype, kind, seed, inst, m, cols, dst, ld, static_cast<cudaStream_t>(stream));
}

}  // extern "C"
