// C ABI of libblockcg.so and the host-side solver drivers.
//
// blockCGrQ (Algorithm 1) runs as a fixed sequence of kernel launches per
// iteration, all on the caller's stream and all gated by a device status
// word, so the host enqueues `check_every` iterations at a time and reads the
// status only between such chunks:
//
//   T  = D_oe P                        stencil            (Sec. 6.2)
//   AP = m^2 P - D_eo T                stencil + epilogue (Sec. 3.2)
//   H  = P^dag AP                      Gram               (Sec. 6.4)
//   beta = H^-1, BC = beta C           dense              (Algorithm 1)
//   W  = Q - AP beta and W^dag W       streaming + Gram in one pass (6.3, 6.4)
//   W^dag W = S^dag S, C = S C, res    dense              (Algorithm 2)
//   Q = W S^-1, X += P BC, P = Q + P S^dag       one fused streaming pass
//   [reliable update, gated]           Algorithm 3:
//      Y += X, X = 0; R = B - A Y; R = Q C (thin QR); S = C C_old^-1;
//      P = Q + P S^dag
//
// The reliable update also serves as the convergence test: when the
// iterated residual meets tol, the true residual of Y decides.  Updates run
// in double-float (native FP64 in the F64_NATIVE form); a convergence they
// report is confirmed once in native FP64 before the solve ends.
#include <cuda_runtime.h>
#include <unistd.h>

#include <cmath>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <map>
#include <mutex>
#include <string>
#include <vector>

#include "../../include/blockcg.h"
#include "internal.h"

using namespace bcg;

struct blockcg_ctx {
  Geom g;
  int dims[4];
  double mass;
  blockcg_params p;
  cudaStream_t stream;
  FieldKind fine;    // Y, B, R and the true-residual operator: native FP64
  FieldKind ru;      // a cheaper kind for the early reliable updates (Algorithm 3)
                     // of a single solve: double-float, or FP64 (= fine: none)
  FieldKind sloppy;  // P, Q, AP, T and the iteration's operator
  FieldKind upd;     // X, the iterated solution update between reliable updates
  void* gauge;
  size_t gauge_bytes;
  void* links_fine;
  void* links_ru;
  void* links_sloppy;
  bool gauge_loaded;
  char* ws;
  size_t ws_bytes;
  std::string err;
  // instrumentation of the current solve
  long long launches;
  struct Timed {
    cudaEvent_t a, b;
    int fine;
  };
  std::vector<cudaEvent_t> ev_pool;
  std::vector<Timed> ev_pending;
  long long n_st[5];   // timed launches per category (see TL)
  double ms_st[5];
  // autotuned register tile of the stencil, keyed by kind * 128 + N
  std::map<int, int> tuned_R;
  // autotuned shared-memory tiles of the block BLAS (sites per tile of the
  // fused update, the Gram and the fused W update + Gram), same key, packed
  // as upd | gram << 8 | wgram << 16
  std::map<int, int> tuned_blas;
  // persisted tuning cache (blockcg_set_tune_cache): file path and entries
  std::string cache_path;
};

namespace {

const size_t ALIGN = 256;
inline size_t up(size_t x) { return (x + ALIGN - 1) / ALIGN * ALIGN; }

enum MatId { M_H = 0, M_G, M_C, M_CPREV, M_BETA, M_BC, M_SINV, M_SH, M_CINV, M_SHRU, M_K, M_RINV, M_COUNT };

struct Ws {
  // fine-kind fields (native FP64); Bru, Yru, Rru: copies in the kind of the
  // early reliable updates (alias B, Y, R when that kind is FP64)
  void *B, *Y, *R, *Tf, *Bru, *Yru, *Rru;
  // update-kind field
  void* X;
  // sloppy-kind fields
  void *Q, *P, *AP, *Ts;
  double2* partials;
  double2* mats;
  double* bnorm;
  double* tres;  // per-column true relative residual of the last check
  SolverStatus* st;
  double* scal;  // CG scalars: rr, alpha, beta, gamma, alpha / gamma
  int* ierr;
  int nblocks;
  size_t total;
};

Ws carve(const blockcg_ctx* h, int N, char* base) {
  Ws w;
  size_t off = 0;
  auto take = [&](size_t bytes) -> char* {
    char* p = base ? base + off : nullptr;
    off += up(bytes);
    return p;
  };
  // first: the tensor-core stencil's column maxima, at an offset that does
  // not depend on N (Geom::tc_colmax points here once the workspace is set)
  take(64 * sizeof(unsigned));
  size_t nel = (size_t)h->g.Vh * N * 3;
  size_t fb = nel * elem_bytes(h->fine), rb = nel * elem_bytes(h->ru),
         sb = nel * elem_bytes(h->sloppy);
  w.B = take(fb);
  w.Y = take(fb);
  w.X = take(nel * elem_bytes(h->upd));
  w.R = take(fb);
  w.Tf = take(fb);  // odd-site temporary of both reliable-update kinds (16-byte elements)
  const bool cheap = h->ru != h->fine;
  w.Bru = cheap ? take(rb) : w.B;
  w.Yru = cheap ? take(rb) : w.Y;
  w.Rru = cheap ? take(rb) : w.R;
  w.Q = take(sb);
  w.P = take(sb);
  w.AP = take(sb);
  w.Ts = (h->sloppy == h->fine) ? w.Tf : take(sb);
  w.nblocks = gram_blocks(N, 3 * h->g.Vh);
  int nb_cg = 2 * 152;
  size_t np = (size_t)(w.nblocks > nb_cg ? w.nblocks : nb_cg) * N * N;
  w.partials = (double2*)take(np * sizeof(double2));
  w.mats = (double2*)take((size_t)M_COUNT * N * N * sizeof(double2));
  w.bnorm = (double*)take(N * sizeof(double));
  w.tres = (double*)take(N * sizeof(double));
  w.st = (SolverStatus*)take(sizeof(SolverStatus));
  w.scal = (double*)take(8 * sizeof(double));
  w.ierr = (int*)take(sizeof(int));
  w.total = off;
  return w;
}

inline double2* mat(const Ws& w, int id, int N) { return w.mats + (size_t)id * N * N; }

blockcg_status fail(blockcg_ctx* h, blockcg_status s, const std::string& msg) {
  if (h) h->err = msg;
  return s;
}

blockcg_status cuda_fail(blockcg_ctx* h, cudaError_t e, const char* where) {
  return fail(h, BLOCKCG_ERR_CUDA, std::string(where) + ": " + cudaGetErrorString(e));
}

#define CK(call)                                       \
  do {                                                 \
    cudaError_t e_ = (call);                           \
    if (e_ != cudaSuccess) return cuda_fail(h, e_, #call); \
  } while (0)

// a kernel launch: checked and counted
#define KL(call)     \
  do {               \
    ++h->launches;   \
    CK(call);        \
  } while (0)

// two timing events destroyed on every return path
struct EventPair {
  cudaEvent_t a = nullptr, b = nullptr;
  cudaError_t create() {
    cudaError_t e = cudaEventCreate(&a);
    return e != cudaSuccess ? e : cudaEventCreate(&b);
  }
  ~EventPair() {
    if (a) cudaEventDestroy(a);
    if (b) cudaEventDestroy(b);
  }
};

cudaEvent_t pool_event(blockcg_ctx* h) {
  if (!h->ev_pool.empty()) {
    cudaEvent_t e = h->ev_pool.back();
    h->ev_pool.pop_back();
    return e;
  }
  cudaEvent_t e = nullptr;
  cudaEventCreate(&e);
  return e;
}

// a launch of category cat, event-timed when params.profile is set:
// 0 iteration stencil, 1 full-precision stencil, 2 Gram, 3 streaming BLAS,
// 4 dense N x N
enum { TC_STENCIL = 0, TC_STENCIL_FINE = 1, TC_GRAM = 2, TC_STREAM = 3, TC_DENSE = 4 };
#define TL(cat_, call)                                        \
  do {                                                        \
    if (h->p.profile) {                                       \
      blockcg_ctx::Timed t_{pool_event(h), pool_event(h), (cat_)}; \
      CK(cudaEventRecord(t_.a, h->stream));                   \
      KL(call);                                               \
      CK(cudaEventRecord(t_.b, h->stream));                   \
      h->ev_pending.push_back(t_);                            \
    } else {                                                  \
      KL(call);                                               \
    }                                                         \
  } while (0)
#define SL(fine_, call) TL((fine_) ? TC_STENCIL_FINE : TC_STENCIL, call)

// after a synchronisation: fold the finished stencil timings into the totals
void drain_events(blockcg_ctx* h) {
  for (auto& t : h->ev_pending) {
    float ms = 0.f;
    if (cudaEventElapsedTime(&ms, t.a, t.b) == cudaSuccess) {
      h->n_st[t.fine] += 1;
      h->ms_st[t.fine] += ms;
    }
    h->ev_pool.push_back(t.a);
    h->ev_pool.push_back(t.b);
  }
  h->ev_pending.clear();
}

void reset_instrumentation(blockcg_ctx* h) {
  h->launches = 0;
  for (int i = 0; i < 5; ++i) {
    h->n_st[i] = 0;
    h->ms_st[i] = 0.0;
  }
  h->ev_pending.clear();
}

void fill_stats(const blockcg_ctx* h, blockcg_stats* st) {
  st->launches = h->launches;
  st->n_stencil = h->n_st[0];
  st->ms_stencil = h->ms_st[0];
  st->n_stencil_fine = h->n_st[1];
  st->ms_stencil_fine = h->ms_st[1];
  st->ms_gram = h->ms_st[TC_GRAM];
  st->ms_stream = h->ms_st[TC_STREAM];
  st->ms_dense = h->ms_st[TC_DENSE];
}

int tile_R(int N) { return N >= 8 ? 4 : (N >= 2 ? 2 : 1); }

// ---- persisted tuning cache --------------------------------------------
// A JSON object with one "key": integer entry per line, shared by every
// handle that names the same file; keys carry the lattice, storage kind or
// precision form, width and the device name, so one file can serve several
// problems and GPUs.  Reads and writes are serialised within the process and
// a write replaces the file atomically (temporary file + rename).
std::mutex g_cache_mutex;

std::string device_tag() {
  int dev = 0;
  cudaDeviceProp prop;
  if (cudaGetDevice(&dev) != cudaSuccess || cudaGetDeviceProperties(&prop, dev) != cudaSuccess) {
    cudaGetLastError();
    return "unknown";
  }
  std::string n = prop.name;
  for (char& c : n)
    if (c == ' ' || c == '"' || c == '\\') c = '_';
  return n;
}

std::map<std::string, long long> cache_read(const std::string& path) {
  std::map<std::string, long long> m;
  FILE* f = fopen(path.c_str(), "r");
  if (!f) return m;
  char line[1024];
  while (fgets(line, sizeof(line), f)) {
    const char* q0 = strchr(line, '"');
    if (!q0) continue;
    const char* q1 = strchr(q0 + 1, '"');
    if (!q1) continue;
    const char* colon = strchr(q1, ':');
    if (!colon) continue;
    char* end = nullptr;
    long long v = strtoll(colon + 1, &end, 10);
    if (end == colon + 1) continue;
    m[std::string(q0 + 1, q1)] = v;
  }
  fclose(f);
  return m;
}

bool cache_write(const std::string& path, const std::map<std::string, long long>& m) {
  std::string tmp = path + ".tmp" + std::to_string((long long)getpid());
  FILE* f = fopen(tmp.c_str(), "w");
  if (!f) return false;
  fprintf(f, "{\n");
  size_t i = 0;
  for (const auto& kv : m) {
    fprintf(f, "  \"%s\": %lld%s\n", kv.first.c_str(), kv.second, ++i < m.size() ? "," : "");
  }
  fprintf(f, "}\n");
  bool ok = fclose(f) == 0;
  if (ok) ok = rename(tmp.c_str(), path.c_str()) == 0;
  if (!ok) remove(tmp.c_str());
  return ok;
}

// value of key in the handle's cache file (false when absent or no file)
bool cache_get(const blockcg_ctx* h, const std::string& key, long long* v) {
  if (h->cache_path.empty()) return false;
  std::lock_guard<std::mutex> lock(g_cache_mutex);
  auto m = cache_read(h->cache_path);
  auto it = m.find(key);
  if (it == m.end()) return false;
  *v = it->second;
  return true;
}

void cache_put(const blockcg_ctx* h, const std::string& key, long long v) {
  if (h->cache_path.empty()) return;
  std::lock_guard<std::mutex> lock(g_cache_mutex);
  auto m = cache_read(h->cache_path);
  m[key] = v;
  cache_write(h->cache_path, m);
}

std::string dims_tag(const blockcg_ctx* h) {
  char buf[64];
  snprintf(buf, sizeof(buf), "%d.%d.%d.%d", h->dims[0], h->dims[1], h->dims[2], h->dims[3]);
  return buf;
}

std::string stencil_key(const blockcg_ctx* h, FieldKind k, int N, int rf) {
  char buf[160];
  snprintf(buf, sizeof(buf), "stencil/%s/kind%d/N%d/recon%d/%s", dims_tag(h).c_str(), (int)k, N,
           rf ? 1 : 0, device_tag().c_str());
  return buf;
}

// Register tile of the stencil for (kind, N): tuned once per handle by timing
// every candidate R on the handle's own buffers (the register-tile tuning of
// Sec. 6.2); in is read, out is scratch.  Falls back to tile_R on any error.
// the stencil flag of a kind's links: two-row storage for the iteration's
// links when params.link_recon is set (the FP64 links are always complete)
int recon_flag(const blockcg_ctx* h, FieldKind k) {
  return (h->p.link_recon && k == h->sloppy && h->sloppy != h->fine && h->sloppy != h->ru)
             ? DSLASH_RECON
             : 0;
}

// Autotuned stencil choice for (kind, N), cached.  Each candidate is timed
// over 3 launches of out = D in; with out2 the candidate is timed on the pair
// the normal operator runs (out = D_oe in, then out2 = m^2 in - D_eo out), so
// that a kernel whose fused epilogue is slow is not chosen on the first half
// alone.
int stencil_R(blockcg_ctx* h, FieldKind k, int N, const void* links, const void* in, void* out,
              void* out2 = nullptr) {
  const int rf = recon_flag(h, k);
  if (h->p.dslash_variant) return h->p.dslash_variant | rf;
  const int key = (int)k * 128 + N;
  auto it = h->tuned_R.find(key);
  if (it != h->tuned_R.end()) return it->second;
  {
    long long v = 0;
    if (cache_get(h, stencil_key(h, k, N, rf), &v)) {
      h->tuned_R[key] = (int)v;
      return (int)v;
    }
  }
  int best = tile_R(N) | rf;
  float best_ms = 1e30f;
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  if (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess) {
    h->tuned_R[key] = best;
    return best;
  }
  Gate g0{nullptr, GATE_ALWAYS};
  const int cands[13] = {1, 2, 4, 8, 1 | DSLASH_TMA, 2 | DSLASH_TMA, 4 | DSLASH_TMA, 8 | DSLASH_TMA,
                         1 | DSLASH_ASYNC, 2 | DSLASH_ASYNC, 4 | DSLASH_ASYNC, 8 | DSLASH_ASYNC,
                         1 | DSLASH_TC};
  for (int R : cands) {
    if ((R & 0xff) > 1 && (R & 0xff) > N) continue;
    // the tensor-core stencil: double-float, FP16 and bfloat16 with N = 16 or
    // 32 and full links only
    if ((R & DSLASH_TC) &&
        (rf || !((k == FK_DF && dslash_tc_supported(h->g, N)) ||
                 ((k == FK_H16 || k == FK_BF16) && dslash_tc16_supported(N)))))
      continue;
    if (rf) {  // two-row links: the plain kernel only
      if (R & (DSLASH_TMA | DSLASH_ASYNC)) continue;
      R |= rf;
    }
    // double-float with N >= 2: the cp.async kernel only.  Timed alone the
    // plain kernel looks up to 4 % faster, but inside the solve (between the
    // Gram, N x N and update kernels) it ran 12-15 % slower than that timing
    // in repeated 32^4 N = 16 measurements, while the cp.async kernel ran as
    // timed.
    if (k == FK_DF && N >= 2 && !(R & (DSLASH_ASYNC | DSLASH_TC))) continue;
    const double m2 = h->mass * h->mass;
    auto run = [&]() {
      cudaError_t e = dslash(k, R, EPI_NONE, links, in, out, nullptr, nullptr, 0.0, h->g, 1, N, g0,
                             h->stream);
      if (e == cudaSuccess && out2)
        e = dslash(k, R, EPI_NORMAL, links, out, out2, in, nullptr, m2, h->g, 0, N, g0, h->stream);
      return e;
    };
    if (run() != cudaSuccess) {
      cudaGetLastError();
      continue;
    }
    cudaEventRecord(e0, h->stream);
    for (int i = 0; i < 3; ++i) run();
    cudaEventRecord(e1, h->stream);
    if (cudaEventSynchronize(e1) != cudaSuccess) continue;
    float ms = 0.f;
    cudaEventElapsedTime(&ms, e0, e1);
    if (ms < best_ms) {
      best_ms = ms;
      best = R;
    }
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  cudaGetLastError();
  h->tuned_R[key] = best;
  cache_put(h, stencil_key(h, k, N, rf), best);
  return best;
}

// sites-per-tile choices of the block BLAS for (kind, N), packed as above
struct BlasTiles {
  int upd, gram, wgram;
};
// packed: update tile in bits 0..7 (UPD_TC as bit 24), Gram tile in bits
// 8..15 (GR_TC as bit 26), fused W + Gram tile in bits 16..23 (WG_TC as
// bit 25)
BlasTiles unpack_tiles(int v) {
  return {(v & 0xff) | ((v >> 24) & 1 ? UPD_TC : 0), ((v >> 8) & 0xff) | ((v >> 26) & 1 ? GR_TC : 0),
          ((v >> 16) & 0xff) | ((v >> 25) & 1 ? WG_TC : 0)};
}
int pack_tiles(const BlasTiles& t) {
  return (t.upd & 0xff) | ((t.upd & UPD_TC) ? 1 << 24 : 0) | ((t.gram & 0xff) << 8) |
         ((t.gram & GR_TC) ? 1 << 26 : 0) | ((t.wgram & 0xff) << 16) |
         ((t.wgram & WG_TC) ? 1 << 25 : 0);
}

BlasTiles cached_tiles(const blockcg_ctx* h, FieldKind k, int N) {
  auto it = h->tuned_blas.find((int)k * 128 + N);
  return it != h->tuned_blas.end() ? unpack_tiles(it->second) : BlasTiles{0, 0, 0};
}

std::string blas_key(const blockcg_ctx* h, FieldKind k, int N) {
  char buf[160];
  snprintf(buf, sizeof(buf), "blas/%s/kind%d/N%d/%s", dims_tag(h).c_str(), (int)k, N,
           device_tag().c_str());
  return buf;
}

// Shared-memory tile sizes of the iteration's block BLAS (the streaming and
// reduction multi-BLAS tile of Sec. 6.3/6.4, which the paper sizes by hand):
// each candidate is timed over 3 launches on buffers that hold no state at
// this point of a solve (AP and the odd temporary stand in for the blocks, R
// for X, the partials buffer receives the Grams), the fastest kept per
// (kind, N) and in the tuning cache.
void tune_blas(blockcg_ctx* h, const Ws& w, int N) {
  const FieldKind k = h->sloppy;
  const int key = (int)k * 128 + N;
  if (h->tuned_blas.count(key)) return;
  long long cv = 0;
  if (cache_get(h, blas_key(h, k, N), &cv)) {
    h->tuned_blas[key] = (int)cv;
    return;
  }
  EventPair ev;
  if (ev.create() != cudaSuccess) {
    cudaGetLastError();
    h->tuned_blas[key] = 0;
    return;
  }
  cudaStream_t s = h->stream;
  Gate g0{nullptr, GATE_ALWAYS};
  const int Vh = h->g.Vh;
  auto time3 = [&](auto&& launch) -> float {
    if (launch() != cudaSuccess) {
      cudaGetLastError();
      return 1e30f;
    }
    cudaEventRecord(ev.a, s);
    for (int i = 0; i < 3; ++i) launch();
    cudaEventRecord(ev.b, s);
    float ms = 1e30f;
    if (cudaEventSynchronize(ev.b) != cudaSuccess || cudaEventElapsedTime(&ms, ev.a, ev.b) != cudaSuccess) {
      cudaGetLastError();
      return 1e30f;
    }
    return ms;
  };
  int best_upd = 0, best_gram = 0, best_wgram = 0;
  float t_upd = 1e30f, t_gram = 1e30f, t_wgram = 1e30f;
  const bool float_kind = (k == FK_F32 || k == FK_H16 || k == FK_BF16);
  for (int variant = 0; variant < 4; ++variant) {
    const bool two_rows = variant & 1, x_global = variant & 2;
    if ((two_rows || x_global) && !float_kind) continue;
    for (int ts : {4, 8, 16, 32}) {
      const int tile = ts | (two_rows ? UPD_TWO_ROWS : 0) | (x_global ? UPD_X_GLOBAL : 0);
      float t = time3([&] {
        return bcg_update(k, h->upd, w.AP, w.Ts, w.R, mat(w, M_SINV, N), mat(w, M_BC, N),
                          mat(w, M_SH, N), N, Vh, g0, s, tile);
      });
      if (t < t_upd) t_upd = t, best_upd = tile;
    }
  }
  if (bcg_update_tc_supported(k, h->upd, N)) {
    float t = time3([&] {
      return bcg_update(k, h->upd, w.AP, w.Ts, w.R, mat(w, M_SINV, N), mat(w, M_BC, N),
                        mat(w, M_SH, N), N, Vh, g0, s, UPD_TC);
    });
    if (t < t_upd) t_upd = t, best_upd = UPD_TC;
  }
  int base = 256 / N;
  if (base < 1) base = 1;
  for (int ts : {base, 2 * base, 4 * base}) {
    if (ts > 255) continue;
    float t = time3([&] {
      return gram_partials(k, w.AP, w.Ts, N, Vh, 1, w.partials, w.nblocks, g0, s, ts);
    });
    if (t < t_gram) t_gram = t, best_gram = ts;
    t = time3([&] {
      return w_update_gram(k, w.AP, w.Ts, mat(w, M_BETA, N), N, Vh, w.partials, w.nblocks, g0, s, ts);
    });
    if (t < t_wgram) t_wgram = t, best_wgram = ts;
  }
  if (w_gram_tc_supported(k, N)) {
    float t = time3([&] {
      return w_update_gram(k, w.AP, w.Ts, mat(w, M_BETA, N), N, Vh, w.partials, w.nblocks, g0, s,
                           WG_TC);
    });
    if (t < t_wgram) t_wgram = t, best_wgram = WG_TC;
    t = time3([&] {
      return gram_partials(k, w.AP, w.Ts, N, Vh, 1, w.partials, w.nblocks, g0, s, GR_TC);
    });
    if (t < t_gram) t_gram = t, best_gram = GR_TC;
  }
  const int packed = pack_tiles({best_upd, best_gram, best_wgram});
  h->tuned_blas[key] = packed;
  cache_put(h, blas_key(h, k, N), packed);
}

int cached_R(const blockcg_ctx* h, FieldKind k, int N) {
  const int rf = recon_flag(h, k);
  if (h->p.dslash_variant) return h->p.dslash_variant | rf;
  auto it = h->tuned_R.find((int)k * 128 + N);
  return it != h->tuned_R.end() ? it->second : (tile_R(N) | rf);
}

blockcg_status check_ready(blockcg_ctx* h, int N) {
  if (!h) return BLOCKCG_ERR_ARG;
  if (N < 1 || N > 64) return fail(h, BLOCKCG_ERR_ARG, "n_rhs must be in [1, 64]");
  if (!h->gauge_loaded) return fail(h, BLOCKCG_ERR_NOMEM, "gauge field not loaded");
  if (!h->ws) return fail(h, BLOCKCG_ERR_NOMEM, "no workspace set");
  if (carve(h, N, nullptr).total > h->ws_bytes)
    return fail(h, BLOCKCG_ERR_NOMEM, "workspace too small for n_rhs");
  return BLOCKCG_OK;
}

FieldKind op_kind(const blockcg_ctx* h) { return h->sloppy; }
const void* op_links(const blockcg_ctx* h) { return h->links_sloppy; }

// A applied to an internal even-site block: out = m^2 in - D_eo D_oe in
blockcg_status apply_A_internal(blockcg_ctx* h, FieldKind k, const void* links, const void* in,
                                void* tmp_odd, void* out, int N, Gate gate) {
  int R = stencil_R(h, k, N, links, in, tmp_odd, out);
  double m2 = h->mass * h->mass;
  KL(dslash(k, R, EPI_NONE, links, in, tmp_odd, nullptr, nullptr, 0.0, h->g, 1, N, gate, h->stream));
  KL(dslash(k, R, EPI_NORMAL, links, tmp_odd, out, in, nullptr, m2, h->g, 0, N, gate, h->stream));
  return BLOCKCG_OK;
}

blockcg_status read_status(blockcg_ctx* h, const Ws& w, SolverStatus* out) {
  CK(cudaMemcpyAsync(out, w.st, sizeof(SolverStatus), cudaMemcpyDeviceToHost, h->stream));
  CK(cudaStreamSynchronize(h->stream));
  drain_events(h);
  return BLOCKCG_OK;
}

int default_check_every(const blockcg_ctx* h, int N) {
  if (h->p.check_every > 0) return h->p.check_every;
  double work = (double)h->g.Vh * N;
  int c = (int)(4.0e6 / work);
  if (c < 1) c = 1;
  if (c > 32) c = 32;
  return c;
}

// R = B - A Y, thin QR, restart of Q and P (Algorithm 3; init: Algorithm 1 set-up)
// The residual R = B - A Y of a restart (Y += X first, unless skip_acc).
// cheap: in the early-update kind (double-float, from a rounded copy of Y;
// accurate to ~2^-48 |A| |Y|, far below residuals well above tol), a
// convergence it reports awaiting FP64 confirmation; otherwise native FP64.
// Y itself is always FP64.
blockcg_status restart_residual(blockcg_ctx* h, const Ws& w, int N, double tol, int init,
                                Gate gate, bool cheap, bool skip_acc) {
  const FieldKind rk = cheap ? h->ru : h->fine;
  const void* links = cheap ? h->links_ru : h->links_fine;
  void* Yk = cheap ? w.Yru : w.Y;
  void* Rk = cheap ? w.Rru : w.R;
  void* Bk = cheap ? w.Bru : w.B;
  int R = cached_R(h, rk, N);
  double m2 = h->mass * h->mass;
  size_t nel = (size_t)h->g.Vh * N * 3;
  cudaStream_t s = h->stream;
  if (!skip_acc) TL(TC_STREAM, accumulate(h->fine, h->upd, w.Y, w.X, nel, gate, s));
  if (cheap) TL(TC_STREAM, convert_field(h->fine, rk, w.Y, Yk, nel, nullptr, gate, s));
  SL(1, dslash(rk, R, EPI_NONE, links, Yk, w.Tf, nullptr, nullptr, 0.0, h->g, 1, N, gate, s));
  SL(1, dslash(rk, R, EPI_RESIDUAL, links, w.Tf, Rk, Yk, Bk, m2, h->g, 0, N, gate, s));
  TL(TC_GRAM, gram_partials(rk, Rk, Rk, N, h->g.Vh, 1, w.partials, w.nblocks, gate, s));
  TL(TC_GRAM, gram_reduce(w.partials, w.nblocks, N, 1, mat(w, M_G, N), gate, s));
  TL(TC_DENSE, dense_restart(mat(w, M_G, N), mat(w, M_C, N), mat(w, M_CPREV, N), mat(w, M_CINV, N),
                   mat(w, M_SHRU, N), w.bnorm, w.tres, tol, init, cheap ? 0 : 1, N, w.st, gate, s));
  TL(TC_STREAM, restart_update(rk, h->sloppy, Rk, w.Q, w.P, mat(w, M_CINV, N), mat(w, M_SHRU, N), init,
                    N, h->g.Vh, gate, s));
  return BLOCKCG_OK;
}

// Early reliable updates use the cheap (double-float) residual while the
// iterated residual of that iteration is above this factor times tol and no
// FP64 confirmation has failed.  The double-float residual's error (~2^-48
// |A| |Y|, about 1e-12 |b| on the 32^4, m = 0.01 workload) has to stay small
// against the residual relative to the rounding of the iteration's storage:
// 2^-24 for FP32 and double-float iterations (factor 1e4), 2^-11 or 2^-8
// for the 16-bit ones (factor 100).
double cheap_ru_above(const blockcg_ctx* h) {
  return (h->sloppy == FK_H16 || h->sloppy == FK_BF16) ? 1e2 : 1e4;
}

// A reliable update (Algorithm 3) gated by `gate`: with a cheaper kind, two
// residual blocks gated on this iteration's residual (GATE_RU_CHEAP /
// GATE_RU_FINE, exactly one of them runs); otherwise the FP64 one.
// The cheap updates pay only where the FP64 stencil is expensive: on small
// problems (V/2 x N below 2^21 site-columns) the extra gated-off launches of
// a second update block cost more per iteration than the cheap updates save.
bool use_cheap_ru(const blockcg_ctx* h, int N) {
  return h->ru != h->fine && (double)h->g.Vh * N >= (double)(1 << 21);
}

blockcg_status restart_block(blockcg_ctx* h, const Ws& w, int N, double tol, int init, Gate gate) {
  if (!use_cheap_ru(h, N) || gate.mode != GATE_RU)
    return restart_residual(h, w, N, tol, init, gate, false, false);
  const size_t nel = (size_t)h->g.Vh * N * 3;
  TL(TC_STREAM, accumulate(h->fine, h->upd, w.Y, w.X, nel, gate, h->stream));
  const double thr = cheap_ru_above(h) * tol;
  blockcg_status rc = restart_residual(h, w, N, tol, init, Gate{gate.st, GATE_RU_CHEAP, thr}, true, true);
  if (rc) return rc;
  return restart_residual(h, w, N, tol, init, Gate{gate.st, GATE_RU_FINE, thr}, false, true);
}

// The true residual of the current Y in native FP64 (R = B - A Y with the
// FP64 links and B), per-column norms against tol.  Confirms a convergence
// that a double-float reliable update reported (done stays set, verified =
// 1), or clears done and sets fp64_only, after which the solve's reliable
// updates are all native FP64 (dense_verify).  Buffers: Tf (odd half) and R.
blockcg_status verify_fp64(blockcg_ctx* h, const Ws& w, int N, double tol) {
  const int R = cached_R(h, FK_F64, N);
  const double m2 = h->mass * h->mass;
  cudaStream_t s = h->stream;
  Gate g0{nullptr, GATE_ALWAYS};
  SL(1, dslash(FK_F64, R, EPI_NONE, h->links_fine, w.Y, w.Tf, nullptr, nullptr, 0.0, h->g, 1, N, g0, s));
  SL(1, dslash(FK_F64, R, EPI_RESIDUAL, h->links_fine, w.Tf, w.R, w.Y, w.B, m2, h->g, 0, N, g0, s));
  TL(TC_GRAM, gram_partials(FK_F64, w.R, w.R, N, h->g.Vh, 1, w.partials, w.nblocks, g0, s));
  TL(TC_GRAM, gram_reduce(w.partials, w.nblocks, N, 1, mat(w, M_K, N), g0, s));
  TL(TC_DENSE, dense_verify(mat(w, M_K, N), w.bnorm, w.tres, tol, N, w.st, s));
  return BLOCKCG_OK;
}

blockcg_status iterate_block(blockcg_ctx* h, const Ws& w, int N, double tol) {
  Gate ga{w.st, GATE_ACTIVE};
  Gate gr{w.st, GATE_RU};
  int R = cached_R(h, h->sloppy, N);
  double m2 = h->mass * h->mass;
  cudaStream_t s = h->stream;
  FieldKind k = h->sloppy;
  SL(0, dslash(k, R, EPI_NONE, h->links_sloppy, w.P, w.Ts, nullptr, nullptr, 0.0, h->g, 1, N, ga, s));
  SL(0, dslash(k, R, EPI_NORMAL, h->links_sloppy, w.Ts, w.AP, w.P, nullptr, m2, h->g, 0, N, ga, s));
  const BlasTiles bt = cached_tiles(h, k, N);
  TL(TC_GRAM, gram_partials(k, w.P, w.AP, N, h->g.Vh, 1, w.partials, w.nblocks, ga, s, bt.gram));
  TL(TC_GRAM, gram_reduce(w.partials, w.nblocks, N, 1, mat(w, M_H, N), ga, s));
  TL(TC_DENSE, dense_beta(mat(w, M_H, N), mat(w, M_C, N), mat(w, M_BETA, N), mat(w, M_BC, N), N, w.st, ga, s));
  // W = Q - AP beta (over Q) with the partials of W^dag W in the same pass
  TL(TC_STREAM, w_update_gram(k, w.Q, w.AP, mat(w, M_BETA, N), N, h->g.Vh, w.partials, w.nblocks,
                              ga, s, bt.wgram));
  TL(TC_GRAM, gram_reduce(w.partials, w.nblocks, N, 1, mat(w, M_G, N), ga, s));
  QrStepParams qp{tol, h->p.ru_delta, h->p.ru_every, h->p.max_iter};
  TL(TC_DENSE, dense_qr_step(mat(w, M_G, N), mat(w, M_C, N), mat(w, M_CPREV, N), mat(w, M_SINV, N),
                   mat(w, M_SH, N), w.bnorm, qp, N, w.st, ga, s));
  TL(TC_STREAM, bcg_update(k, h->upd, w.Q, w.P, w.X, mat(w, M_SINV, N), mat(w, M_BC, N), mat(w, M_SH, N), N,
                h->g.Vh, ga, s, bt.upd));
  return restart_block(h, w, N, tol, 0, gr);
}

blockcg_status status_to_result(blockcg_ctx* h, const SolverStatus& st) {
  if (st.error) {
    const char* what = blockcg_status_string((blockcg_status)st.error);
    return fail(h, (blockcg_status)st.error, std::string("device reported: ") + what);
  }
  return BLOCKCG_OK;
}

blockcg_status check_solve_args(blockcg_ctx* h, const void* B, const void* X, int n_rhs,
                                double tol) {
  blockcg_status rc = check_ready(h, n_rhs);
  if (rc) return rc;
  if (!B || !X) return fail(h, BLOCKCG_ERR_ARG, "null pointer");
  if (!(tol > 0) || !std::isfinite(tol)) return fail(h, BLOCKCG_ERR_ARG, "tol must be > 0");
  return BLOCKCG_OK;
}

// autotune the stencils a block solve of width N uses (no-op once cached)
// (after the set-up: P and Y hold data; AP, Ts, R and Tf are free until the
// first iteration and the next reliable update rewrite them)
void tune_block(blockcg_ctx* h, const Ws& w, int N) {
  tune_blas(h, w, N);
  stencil_R(h, h->sloppy, N, h->links_sloppy, w.P, w.Ts, w.AP);
  stencil_R(h, h->fine, N, h->links_fine, w.Y, w.Tf, w.R);
  if (use_cheap_ru(h, N)) stencil_R(h, h->ru, N, h->links_ru, w.Yru, w.Tf, w.Rru);
}

// Algorithm 1 set-up: B and X in internal layout, |b_i|, X = 0 (update),
// P = 0, and the initial R = B - A Y, thin QR and P = Q (an ungated restart)
blockcg_status solve_begin(blockcg_ctx* h, const Ws& w, const void* B, const void* X, int N,
                           double tol) {
  cudaStream_t s = h->stream;
  size_t nel = (size_t)h->g.Vh * N * 3;
  Gate g0{nullptr, GATE_ALWAYS};
  Gate ga{w.st, GATE_ACTIVE};
  CK(cudaMemsetAsync(w.st, 0, sizeof(SolverStatus), s));
  CK(cudaMemsetAsync(w.tres, 0xff, N * sizeof(double), s));  // NaN until a true residual exists
  KL(to_internal(h->fine, (const double2*)B, w.B, N, h->g.Vh, s));
  if (w.Bru != w.B) KL(to_internal(h->ru, (const double2*)B, w.Bru, N, h->g.Vh, s));
  KL(to_internal(h->fine, (const double2*)X, w.Y, N, h->g.Vh, s));
  CK(zero_field(h->upd, w.X, nel, s));
  CK(zero_field(h->sloppy, w.P, nel, s));
  KL(gram_partials(h->fine, w.B, w.B, N, h->g.Vh, 1, w.partials, w.nblocks, g0, s));
  KL(gram_reduce(w.partials, w.nblocks, N, 1, mat(w, M_G, N), g0, s));
  KL(dense_bnorm(mat(w, M_G, N), w.bnorm, N, w.st, s));
  return restart_block(h, w, N, tol, 1, ga);
}

// a convergence the solve may report: reported by a native-FP64 reliable
// update, or by a double-float one and confirmed in native FP64
bool converged(const blockcg_ctx* h, const SolverStatus& hs) {
  (void)h;
  return hs.done && hs.verified;
}



// Host-driven iteration from the current device state: enqueue chunks of
// gated iterations and poll the status word between them; a convergence
// reported by a double-float reliable update is checked in native FP64
// (verify_fp64), and if that check fails the iteration goes on.  Returns
// with *hs the last status (converged, error, or the iteration budget spent).
blockcg_status host_loop(blockcg_ctx* h, const Ws& w, int N, double tol, SolverStatus* hs) {
  const int chunk = default_check_every(h, N);
  for (;;) {
    blockcg_status rc = read_status(h, w, hs);
    if (rc) return rc;
    if (hs->error || converged(h, *hs)) return BLOCKCG_OK;
    if (hs->done) {
      rc = verify_fp64(h, w, N, tol);
      if (rc) return rc;
      continue;
    }
    if (hs->iters >= h->p.max_iter || hs->stopped) return BLOCKCG_OK;
    int n = chunk;
    if (hs->iters + n > h->p.max_iter) n = h->p.max_iter - hs->iters;
    if (n <= 0) n = 1;
    for (int i = 0; i < n; ++i) {
      rc = iterate_block(h, w, N, tol);
      if (rc) return rc;
    }
  }
}

// after the iterations: at max_iter fold the last update into Y and take the
// true residual (in native FP64); write Y to the caller's X.  *result = the
// solve's outcome.
blockcg_status solve_end(blockcg_ctx* h, const Ws& w, void* X, int N, double tol,
                         SolverStatus* hs, blockcg_status* result) {
  Gate g0{nullptr, GATE_ALWAYS};
  *result = status_to_result(h, *hs);
  if (!*result && !converged(h, *hs)) {
    blockcg_status rc = hs->done ? verify_fp64(h, w, N, tol) : restart_block(h, w, N, tol, 1, g0);
    if (rc) return rc;
    rc = read_status(h, w, hs);
    if (rc) return rc;
    *result = status_to_result(h, *hs);
    if (!*result && !converged(h, *hs))
      *result = fail(h, BLOCKCG_ERR_NOT_CONVERGED, "max_iter reached");
  }
  KL(from_internal(h->fine, w.Y, (double2*)X, N, h->g.Vh, h->stream));
  return BLOCKCG_OK;
}

}  // namespace

// ===================================================================== ABI

extern "C" {

void blockcg_default_params(blockcg_params* p) {
  if (!p) return;
  p->max_iter = 100000;
  p->ru_delta = 0.1;
  p->ru_every = 0;
  p->prec = BLOCKCG_PREC_F64;
  p->antiperiodic_t = 0;
  p->check_every = 0;
  p->profile = 0;
  p->dslash_variant = 0;
  p->link_recon = 0;
  p->wait_limit_ns = 0;
}

const char* blockcg_status_string(blockcg_status s) {
  switch (s) {
    case BLOCKCG_OK: return "ok";
    case BLOCKCG_ERR_ARG: return "invalid argument";
    case BLOCKCG_ERR_CUDA: return "CUDA error";
    case BLOCKCG_ERR_NOMEM: return "insufficient or missing device buffer";
    case BLOCKCG_ERR_BREAKDOWN: return "Cholesky breakdown (rank-deficient block)";
    case BLOCKCG_ERR_NONFINITE: return "non-finite value in a Gram matrix";
    case BLOCKCG_ERR_NOT_CONVERGED: return "not converged within max_iter";
    case BLOCKCG_ERR_TIMEOUT: return "device wait timed out";
  }
  return "unknown status";
}

const char* blockcg_last_error(blockcg_t h) { return h ? h->err.c_str() : "null handle"; }

blockcg_status blockcg_create(blockcg_t* out, const int dims[4], double mass,
                              const blockcg_params* p, void* stream) {
  if (!out || !dims) return BLOCKCG_ERR_ARG;
  *out = nullptr;
  long long V = 1;
  for (int mu = 0; mu < 4; ++mu) {
    if (dims[mu] < 2 || (dims[mu] & 1)) return BLOCKCG_ERR_ARG;
    V *= dims[mu];
  }
  if (V / 2 >= (1LL << 31) / 64) return BLOCKCG_ERR_ARG;
  if (!std::isfinite(mass)) return BLOCKCG_ERR_ARG;
  blockcg_params prm;
  blockcg_default_params(&prm);
  if (p) prm = *p;
  if (prm.max_iter < 1 || prm.ru_delta < 0 || !(prm.ru_delta < 1) || prm.ru_every < 0 ||
      prm.check_every < 0 || (int)prm.prec < 0 || (int)prm.prec > 4)
    return BLOCKCG_ERR_ARG;
  {
    int r = prm.dslash_variant & ~(DSLASH_TMA | DSLASH_ASYNC | DSLASH_BLOCKED | DSLASH_TC);
    if (prm.dslash_variant != 0 && r != 1 && r != 2 && r != 4 && r != 8) return BLOCKCG_ERR_ARG;
  }
  if (prm.link_recon != 0 && prm.link_recon != 12) return BLOCKCG_ERR_ARG;
  if (prm.wait_limit_ns < 0) return BLOCKCG_ERR_ARG;
  if (prm.link_recon == 12 && prm.prec != BLOCKCG_PREC_MIXED_F32 &&
      prm.prec != BLOCKCG_PREC_MIXED_F16 && prm.prec != BLOCKCG_PREC_MIXED_BF16)
    return BLOCKCG_ERR_ARG;
  blockcg_ctx* h = new blockcg_ctx();
  for (int mu = 0; mu < 4; ++mu) {
    h->dims[mu] = dims[mu];
    h->g.L[mu] = dims[mu];
  }
  h->g.hx = dims[0] / 2;
  h->g.Vh = (int)(V / 2);
  h->g.antiperiodic = prm.antiperiodic_t ? 1 : 0;
  h->g.inv_c[0] = h->g.inv_c[1] = 0.f;
  h->g.wait_ns = (unsigned long long)prm.wait_limit_ns;
  h->g.tc_colmax = nullptr;
  h->mass = mass;
  h->p = prm;
  h->stream = (cudaStream_t)stream;
  h->fine = FK_F64;
  switch (prm.prec) {
    case BLOCKCG_PREC_F64: h->sloppy = FK_DF; h->upd = FK_DF; break;
    case BLOCKCG_PREC_F64_NATIVE: h->sloppy = FK_F64; h->upd = FK_F64; break;
    case BLOCKCG_PREC_MIXED_F32: h->sloppy = FK_F32; h->upd = FK_DF; break;
    case BLOCKCG_PREC_MIXED_F16: h->sloppy = FK_H16; h->upd = FK_DF; break;
    case BLOCKCG_PREC_MIXED_BF16: h->sloppy = FK_BF16; h->upd = FK_DF; break;
  }
  h->ru = (prm.prec == BLOCKCG_PREC_F64_NATIVE) ? FK_F64 : FK_DF;
  // with 16-bit storage the sloppy recursion can stagnate (bfloat16's 8-bit
  // significand) or drift (FP16 on ill-conditioned problems) before the
  // residual falls by ru_delta; a periodic reliable update keeps it on track
  if ((prm.prec == BLOCKCG_PREC_MIXED_BF16 || prm.prec == BLOCKCG_PREC_MIXED_F16) &&
      h->p.ru_every == 0)
    h->p.ru_every = 10;
  h->gauge = nullptr;
  h->gauge_bytes = 0;
  h->links_fine = h->links_ru = h->links_sloppy = nullptr;
  h->gauge_loaded = false;
  h->ws = nullptr;
  h->ws_bytes = 0;
  reset_instrumentation(h);
  *out = h;
  return BLOCKCG_OK;
}

void blockcg_destroy(blockcg_t h) {
  if (!h) return;
  for (auto& t : h->ev_pending) {
    h->ev_pool.push_back(t.a);
    h->ev_pool.push_back(t.b);
  }
  for (cudaEvent_t e : h->ev_pool) cudaEventDestroy(e);
  delete h;
}

size_t blockcg_gauge_bytes(blockcg_t h) {
  if (!h) return 0;
  size_t b = up(links_bytes(h->fine, h->g));
  if (h->sloppy != h->fine) b += up(links_bytes(h->sloppy, h->g, h->p.link_recon));
  if (h->ru != h->fine && h->ru != h->sloppy) b += up(links_bytes(h->ru, h->g));
  if (h->p.link_recon) b += ALIGN;  // scratch of the link check
  return b;
}

blockcg_status blockcg_load_gauge(blockcg_t h, const void* fat, const void* lng, void* storage,
                                  size_t storage_bytes) {
  if (!h) return BLOCKCG_ERR_ARG;
  if (!fat || !lng || !storage) return fail(h, BLOCKCG_ERR_ARG, "null pointer");
  if (storage_bytes < blockcg_gauge_bytes(h)) return fail(h, BLOCKCG_ERR_NOMEM, "gauge storage too small");
  const int recon = h->p.link_recon;
  if (recon) {
    // two-row storage needs every link to be a real multiple of an SU(3)
    // matrix, one multiple per kind: check on the device and read the scales
    char* scratch = (char*)storage + blockcg_gauge_bytes(h) - ALIGN;
    double* c = (double*)scratch;
    int* bad = (int*)(scratch + 2 * sizeof(double));
    CK(check_scaled_su3((const double2*)fat, (const double2*)lng, 2LL * h->g.Vh, 1e-10, c, bad,
                        h->stream));
    double hc[2];
    int hbad = 1;
    CK(cudaMemcpyAsync(hc, c, sizeof(hc), cudaMemcpyDeviceToHost, h->stream));
    CK(cudaMemcpyAsync(&hbad, bad, sizeof(int), cudaMemcpyDeviceToHost, h->stream));
    CK(cudaStreamSynchronize(h->stream));
    if (hbad || !(hc[0] != 0.0) || !(hc[1] != 0.0))
      return fail(h, BLOCKCG_ERR_ARG,
                  "link_recon = 12 needs every fat and long link to be c U, U in SU(3), "
                  "c one real constant per kind");
    // the packed hop matrices carry a further factor +-1/2 (see Geom)
    h->g.inv_c[0] = (float)(2.0 / hc[0]);
    h->g.inv_c[1] = (float)(2.0 / hc[1]);
  }
  h->gauge = storage;
  h->gauge_bytes = storage_bytes;
  // [FP64 links][iteration links, if another kind][reliable-update links, if
  // a third kind]
  char* next = (char*)storage + up(links_bytes(h->fine, h->g));
  h->links_fine = storage;
  h->links_sloppy = storage;
  if (h->sloppy != h->fine) {
    h->links_sloppy = next;
    next += up(links_bytes(h->sloppy, h->g, recon));
  }
  h->links_ru = (h->ru == h->fine) ? h->links_fine : (h->ru == h->sloppy) ? h->links_sloppy : next;
  CK(pack_links(h->fine, (const double2*)fat, (const double2*)lng, h->links_fine, h->g,
                h->p.antiperiodic_t, 0, h->stream));
  if (h->sloppy != h->fine)
    CK(pack_links(h->sloppy, (const double2*)fat, (const double2*)lng, h->links_sloppy, h->g,
                  h->p.antiperiodic_t, recon, h->stream));
  if (h->links_ru != h->links_fine && h->links_ru != h->links_sloppy)
    CK(pack_links(h->ru, (const double2*)fat, (const double2*)lng, h->links_ru, h->g,
                  h->p.antiperiodic_t, 0, h->stream));
  h->gauge_loaded = true;
  return BLOCKCG_OK;
}

size_t blockcg_workspace_bytes(blockcg_t h, int n_rhs) {
  if (!h || n_rhs < 1 || n_rhs > 64) return 0;
  return carve(h, n_rhs, nullptr).total;
}

blockcg_status blockcg_set_workspace(blockcg_t h, void* ws, size_t bytes) {
  if (!h) return BLOCKCG_ERR_ARG;
  if (!ws || bytes < blockcg_workspace_bytes(h, 1)) return fail(h, BLOCKCG_ERR_NOMEM, "workspace too small");
  if (((uintptr_t)ws) % 16) return fail(h, BLOCKCG_ERR_ARG, "workspace not 16-byte aligned");
  h->ws = (char*)ws;
  h->ws_bytes = bytes;
  h->g.tc_colmax = (unsigned*)ws;  // the first region of carve()
  return BLOCKCG_OK;
}

blockcg_status blockcg_dslash(blockcg_t h, const void* in, void* out, int n_rhs, int out_parity) {
  blockcg_status rc = check_ready(h, n_rhs);
  if (rc) return rc;
  if (!in || !out || (out_parity & ~1)) return fail(h, BLOCKCG_ERR_ARG, "bad argument");
  Ws w = carve(h, n_rhs, h->ws);
  FieldKind k = op_kind(h);
  Gate g0{nullptr, GATE_ALWAYS};
  CK(to_internal(k, (const double2*)in, w.Q, n_rhs, h->g.Vh, h->stream));
  CK(dslash(k, stencil_R(h, k, n_rhs, op_links(h), w.Q, w.AP), EPI_NONE, op_links(h), w.Q, w.AP, nullptr, nullptr, 0.0, h->g,
            out_parity, n_rhs, g0, h->stream));
  CK(from_internal(k, w.AP, (double2*)out, n_rhs, h->g.Vh, h->stream));
  return BLOCKCG_OK;
}

blockcg_status blockcg_apply_MdagM(blockcg_t h, const void* in, void* out, int n_rhs) {
  blockcg_status rc = check_ready(h, n_rhs);
  if (rc) return rc;
  if (!in || !out) return fail(h, BLOCKCG_ERR_ARG, "null pointer");
  Ws w = carve(h, n_rhs, h->ws);
  FieldKind k = op_kind(h);
  Gate g0{nullptr, GATE_ALWAYS};
  CK(to_internal(k, (const double2*)in, w.P, n_rhs, h->g.Vh, h->stream));
  rc = apply_A_internal(h, k, op_links(h), w.P, w.Ts, w.AP, n_rhs, g0);
  if (rc) return rc;
  CK(from_internal(k, w.AP, (double2*)out, n_rhs, h->g.Vh, h->stream));
  return BLOCKCG_OK;
}

blockcg_status blockcg_link_grad(blockcg_t h, const void* X, const void* Lam, int n_rhs,
                                 void* grad_fat, void* grad_long) {
  blockcg_status rc = check_ready(h, n_rhs);
  if (rc) return rc;
  if (!X || !Lam || (!grad_fat && !grad_long)) return fail(h, BLOCKCG_ERR_ARG, "null pointer");
  const int N = n_rhs;
  Ws w = carve(h, N, h->ws);
  cudaStream_t s = h->stream;
  Gate g0{nullptr, GATE_ALWAYS};
  const int R = cached_R(h, h->fine, N);
  // native FP64: B = X, Y = Lam (even); Tf = D_oe X, R = D_oe Lam (odd)
  KL(to_internal(FK_F64, (const double2*)X, w.B, N, h->g.Vh, s));
  KL(to_internal(FK_F64, (const double2*)Lam, w.Y, N, h->g.Vh, s));
  KL(dslash(FK_F64, R, EPI_NONE, h->links_fine, w.B, w.Tf, nullptr, nullptr, 0.0, h->g, 1, N, g0, s));
  KL(dslash(FK_F64, R, EPI_NONE, h->links_fine, w.Y, w.R, nullptr, nullptr, 0.0, h->g, 1, N, g0, s));
  KL(link_grad((const double2*)w.B, (const double2*)w.Y, (const double2*)w.Tf,
               (const double2*)w.R, (double2*)grad_fat, (double2*)grad_long, h->g, N,
               h->p.antiperiodic_t, s));
  return BLOCKCG_OK;
}

blockcg_status blockcg_block_cdot(blockcg_t h, const void* X, const void* Y, int n_rhs, void* K) {
  blockcg_status rc = check_ready(h, n_rhs);
  if (rc) return rc;
  if (!X || !Y || !K) return fail(h, BLOCKCG_ERR_ARG, "null pointer");
  Ws w = carve(h, n_rhs, h->ws);
  FieldKind k = op_kind(h);
  Gate g0{nullptr, GATE_ALWAYS};
  CK(to_internal(k, (const double2*)X, w.Q, n_rhs, h->g.Vh, h->stream));
  CK(to_internal(k, (const double2*)Y, w.P, n_rhs, h->g.Vh, h->stream));
  CK(gram_partials(k, w.Q, w.P, n_rhs, h->g.Vh, 0, w.partials, w.nblocks, g0, h->stream));
  CK(gram_reduce(w.partials, w.nblocks, n_rhs, 0, (double2*)K, g0, h->stream));
  return BLOCKCG_OK;
}

blockcg_status blockcg_block_caxpy(blockcg_t h, const void* X, const void* a, void* Y, int n_rhs) {
  blockcg_status rc = check_ready(h, n_rhs);
  if (rc) return rc;
  if (!X || !a || !Y) return fail(h, BLOCKCG_ERR_ARG, "null pointer");
  Ws w = carve(h, n_rhs, h->ws);
  FieldKind k = op_kind(h);
  CK(to_internal(k, (const double2*)X, w.Q, n_rhs, h->g.Vh, h->stream));
  CK(to_internal(k, (const double2*)Y, w.P, n_rhs, h->g.Vh, h->stream));
  CK(block_caxpy(k, w.Q, (const double2*)a, w.P, n_rhs, h->g.Vh, h->stream));
  CK(from_internal(k, w.P, (double2*)Y, n_rhs, h->g.Vh, h->stream));
  return BLOCKCG_OK;
}

blockcg_status blockcg_thin_qr(blockcg_t h, const void* M, void* Q, void* R, int n_rhs) {
  blockcg_status rc = check_ready(h, n_rhs);
  if (rc) return rc;
  if (!M || !Q || !R) return fail(h, BLOCKCG_ERR_ARG, "null pointer");
  Ws w = carve(h, n_rhs, h->ws);
  FieldKind k = op_kind(h);
  Gate g0{nullptr, GATE_ALWAYS};
  int N = n_rhs;
  CK(to_internal(k, (const double2*)M, w.Q, N, h->g.Vh, h->stream));
  CK(gram_partials(k, w.Q, w.Q, N, h->g.Vh, 1, w.partials, w.nblocks, g0, h->stream));
  CK(gram_reduce(w.partials, w.nblocks, N, 1, mat(w, M_H, N), g0, h->stream));
  CK(dense_chol_upper(mat(w, M_H, N), (double2*)R, mat(w, M_RINV, N), N, w.ierr, h->stream));
  CK(block_trmul(k, w.Q, mat(w, M_RINV, N), w.P, N, h->g.Vh, h->stream));
  CK(from_internal(k, w.P, (double2*)Q, N, h->g.Vh, h->stream));
  int err = 0;
  CK(cudaMemcpyAsync(&err, w.ierr, sizeof(int), cudaMemcpyDeviceToHost, h->stream));
  CK(cudaStreamSynchronize(h->stream));
  if (err) return fail(h, (blockcg_status)err, "thin QR: Cholesky failed");
  return BLOCKCG_OK;
}

blockcg_status blockcg_solve(blockcg_t h, const void* B, void* X, int n_rhs, double tol,
                             blockcg_stats* stats) {
  blockcg_status rc = check_solve_args(h, B, X, n_rhs, tol);
  if (rc) return rc;
  const int N = n_rhs;
  Ws w = carve(h, N, h->ws);
  cudaStream_t s = h->stream;
  reset_instrumentation(h);
  EventPair ev;
  CK(ev.create());
  cudaEvent_t e0 = ev.a, e1 = ev.b;
  CK(cudaEventRecord(e0, s));
  rc = solve_begin(h, w, B, X, N, tol);
  if (rc) return rc;
  tune_block(h, w, N);
  SolverStatus hs;
  memset(&hs, 0, sizeof(hs));
  rc = host_loop(h, w, N, tol, &hs);
  if (rc) return rc;
  blockcg_status result = BLOCKCG_OK;
  rc = solve_end(h, w, X, N, tol, &hs, &result);
  if (rc) return rc;
  CK(cudaEventRecord(e1, s));
  CK(cudaEventSynchronize(e1));
  drain_events(h);
  float ms = 0;
  cudaEventElapsedTime(&ms, e0, e1);
  if (stats) {
    stats->iters = hs.iters;
    stats->reliable_updates = hs.reliable_updates;
    stats->true_rel_res_max = hs.true_res_max;
    stats->ms_total = ms;
    fill_stats(h, stats);
    stats->stencil_variant = cached_R(h, h->sloppy, N);
    if (stats->true_rel_res) {
      CK(cudaMemcpyAsync(stats->true_rel_res, w.tres, N * sizeof(double), cudaMemcpyDeviceToHost, s));
      CK(cudaStreamSynchronize(s));
    }
  }
  return result;
}

blockcg_status blockcg_solve_cg(blockcg_t h, const void* B, void* X, int n_rhs, double tol,
                                blockcg_stats* stats) {
  blockcg_status rc = check_ready(h, 1);
  if (rc) return rc;
  if (n_rhs < 1 || n_rhs > 64) return fail(h, BLOCKCG_ERR_ARG, "n_rhs must be in [1, 64]");
  if (!B || !X) return fail(h, BLOCKCG_ERR_ARG, "null pointer");
  if (!(tol > 0) || !std::isfinite(tol)) return fail(h, BLOCKCG_ERR_ARG, "tol must be > 0");
  Ws w = carve(h, 1, h->ws);
  cudaStream_t s = h->stream;
  const int Vh = h->g.Vh;
  const FieldKind fk = h->fine, sk = h->sloppy, xk = h->upd;
  const double m2 = h->mass * h->mass;
  const size_t col = (size_t)Vh * 3;
  // full precision: b, y (solution accumulator), rf (true residual), tf
  // iteration: x (update, kind upd), r, p, Ap, t (sloppy kind)
  void *b = w.B, *y = w.Y, *rf = w.R, *tf = w.Tf;
  void *x = w.X, *r = w.Q, *p = w.P, *Ap = w.AP, *t = w.Ts;
  double* rr = w.scal + 0;
  double* alpha = w.scal + 1;
  double* beta = w.scal + 2;
  double* gam = w.scal + 3;      // scale of the iteration's r and p
  double* alpha_x = w.scal + 4;  // alpha / gamma, the coefficient of the x update
  double2* red = mat(w, M_K, 1);
  int nb_cg = 2 * 152;
  Gate g0{nullptr, GATE_ALWAYS};
  Gate ga{w.st, GATE_ACTIVE};
  Gate gi{w.st, GATE_ITER};
  reset_instrumentation(h);
  EventPair ev;
  CK(ev.create());
  cudaEvent_t e0 = ev.a, e1 = ev.b;
  CK(cudaEventRecord(e0, s));
  int total_iters = 0, total_ru = 0;
  double worst = 0.0;
  blockcg_status result = BLOCKCG_OK;
  const int chunk = default_check_every(h, 1);
  for (int j = 0; j < n_rhs && !result; ++j) {
    CK(cudaMemsetAsync(w.st, 0, sizeof(SolverStatus), s));
    CK(cudaMemsetAsync(w.scal, 0, 8 * sizeof(double), s));
    KL(to_internal(fk, (const double2*)B + j * col, b, 1, Vh, s));
    KL(to_internal(fk, (const double2*)X + j * col, y, 1, Vh, s));
    CK(zero_field(xk, x, col, s));
    CK(zero_field(sk, p, col, s));
    TL(TC_GRAM, gram_partials(fk, b, b, 1, Vh, 1, w.partials, w.nblocks, g0, s));
    TL(TC_GRAM, gram_reduce(w.partials, w.nblocks, 1, 1, red, g0, s));
    KL(dense_bnorm(red, w.bnorm, 1, w.st, s));
    SolverStatus hs;
    memset(&hs, 0, sizeof(hs));
    bool restart = true;
    int launched = 0, n_restart = 0;
    for (;;) {
      if (restart) {
        // reliable update: y += x, x = 0, rf = b - A y in full precision,
        // r = rf in the iteration's precision, then p = r + beta p with beta
        // from the true residual (p = r at the start)
        TL(TC_STREAM, accumulate(fk, xk, y, x, col, ga, s));
        SL(1, dslash(fk, 1, EPI_NONE, h->links_fine, y, tf, nullptr, nullptr, 0.0, h->g, 1, 1, ga, s));
        SL(1, dslash(fk, 1, EPI_RESIDUAL, h->links_fine, tf, rf, y, b, m2, h->g, 0, 1, ga, s));
        TL(TC_GRAM, gram_partials(fk, rf, rf, 1, Vh, 1, w.partials, w.nblocks, ga, s));
        TL(TC_GRAM, gram_reduce(w.partials, w.nblocks, 1, 1, red, ga, s));
        TL(TC_DENSE, cg_restart_check(red, rr, beta, gam, w.bnorm, (double)col, tol,
                                      n_restart == 0, w.st, s));
        TL(TC_STREAM, convert_field(fk, sk, rf, r, col, gam, ga, s));
        TL(TC_STREAM, cg_xpay(sk, p, r, beta, Vh, ga, s));
        restart = false;
        ++n_restart;
      }
      rc = read_status(h, w, &hs);
      if (rc) return rc;
      if (hs.done || hs.error) break;
      if (hs.ru_pending) {  // converged or residual dropped by delta: reliable update
        restart = true;
        continue;
      }
      if (hs.iters >= h->p.max_iter) break;
      int n = chunk;
      if (launched + n > h->p.max_iter) n = h->p.max_iter - launched;
      if (n <= 0) n = 1;
      for (int i = 0; i < n; ++i) {
        SL(0, dslash(sk, 1 | recon_flag(h, sk), EPI_NONE, h->links_sloppy, p, t, nullptr, nullptr, 0.0,
                     h->g, 1, 1, gi, s));
        SL(0, dslash(sk, 1 | recon_flag(h, sk), EPI_NORMAL, h->links_sloppy, t, Ap, p, nullptr, m2,
                     h->g, 0, 1, gi, s));
        TL(TC_GRAM, gram_partials(sk, p, Ap, 1, Vh, 1, w.partials, w.nblocks, gi, s));
        TL(TC_GRAM, gram_reduce(w.partials, w.nblocks, 1, 1, red, gi, s));
        TL(TC_DENSE, cg_scalar_alpha(red, rr, gam, alpha, alpha_x, w.st, gi, s));
        TL(TC_STREAM, cg_axpy_norm(sk, xk, x, r, p, Ap, alpha, alpha_x, w.partials, nb_cg, Vh, gi, s));
        TL(TC_GRAM, gram_reduce(w.partials, nb_cg, 1, 1, red + 1, gi, s));
        TL(TC_DENSE, cg_scalar_beta(red + 1, rr, beta, w.bnorm, gam, tol, h->p.ru_delta, w.st, gi, s));
        TL(TC_STREAM, cg_xpay(sk, p, r, beta, Vh, gi, s));
      }
      launched += n;
    }
    total_iters += hs.iters;
    total_ru += n_restart - 1;
    if (hs.error) result = status_to_result(h, hs);
    else if (!hs.done) {
      // max_iter: fold the update into y for the returned iterate
      TL(TC_STREAM, accumulate(fk, xk, y, x, col, g0, s));
      result = fail(h, BLOCKCG_ERR_NOT_CONVERGED, "max_iter reached");
    }
    if (hs.true_res_max > worst) worst = hs.true_res_max;
    if (stats && stats->true_rel_res) stats->true_rel_res[j] = hs.true_res_max;
    KL(from_internal(fk, y, (double2*)X + j * col, 1, Vh, s));
  }
  CK(cudaEventRecord(e1, s));
  CK(cudaEventSynchronize(e1));
  drain_events(h);
  float ms = 0;
  cudaEventElapsedTime(&ms, e0, e1);
  if (stats) {
    stats->iters = total_iters;
    stats->reliable_updates = total_ru;
    stats->true_rel_res_max = worst;
    stats->ms_total = ms;
    fill_stats(h, stats);
  }
  return result;
}

blockcg_status blockcg_set_tune_cache(blockcg_t h, const char* path) {
  if (!h) return BLOCKCG_ERR_ARG;
  h->cache_path = path ? path : "";
  return BLOCKCG_OK;
}

blockcg_status blockcg_solve_many(blockcg_t h, const void* B, void* X, int m_rhs, double tol,
                                  int width, blockcg_many_stats* st) {
  if (!h) return BLOCKCG_ERR_ARG;
  if (!B || !X) return fail(h, BLOCKCG_ERR_ARG, "null pointer");
  if (m_rhs < 1) return fail(h, BLOCKCG_ERR_ARG, "m_rhs must be >= 1");
  if (width < 0 || width > 64) return fail(h, BLOCKCG_ERR_ARG, "width must be in [0, 64]");
  if (!(tol > 0) || !std::isfinite(tol)) return fail(h, BLOCKCG_ERR_ARG, "tol must be > 0");
  if (!h->ws) return fail(h, BLOCKCG_ERR_NOMEM, "no workspace set");
  int maxw = 64;
  while (maxw > 1 && carve(h, maxw, nullptr).total > h->ws_bytes) --maxw;
  if (carve(h, 1, nullptr).total > h->ws_bytes) return fail(h, BLOCKCG_ERR_NOMEM, "workspace too small");
  if (width > maxw) return fail(h, BLOCKCG_ERR_NOMEM, "width beyond the workspace");
  blockcg_many_stats loc;
  memset(&loc, 0, sizeof(loc));
  if (st) loc.true_rel_res = st->true_rel_res;
  const size_t col_bytes = (size_t)h->g.Vh * 3 * sizeof(double2);
  int done = 0;
  blockcg_status result = BLOCKCG_OK;
  // one block of n columns starting at column done
  auto solve_block = [&](int n, double* ms_out) -> blockcg_status {
    blockcg_stats bs;
    memset(&bs, 0, sizeof(bs));
    bs.true_rel_res = loc.true_rel_res ? loc.true_rel_res + done : nullptr;
    blockcg_status rc = blockcg_solve(h, (const char*)B + done * col_bytes,
                                      (char*)X + done * col_bytes, n, tol, &bs);
    loc.blocks += 1;
    loc.iters_total += bs.iters;
    loc.ms_total += bs.ms_total;
    if (bs.true_rel_res_max > loc.true_rel_res_max || std::isnan(bs.true_rel_res_max))
      loc.true_rel_res_max = bs.true_rel_res_max;
    if (ms_out) *ms_out = bs.ms_total;
    done += n;
    return rc;
  };
  char keybuf[200];
  snprintf(keybuf, sizeof(keybuf), "width/%s/prec%d/m=%.6g/tol=%.3g/ru%d/%s", dims_tag(h).c_str(),
           (int)h->p.prec, h->mass, tol, h->p.ru_every, device_tag().c_str());
  const std::string wkey = keybuf;
  int chosen = width;
  if (chosen == 0) {
    long long v = 0;
    if (cache_get(h, wkey, &v) && v >= 1 && v <= maxw) {
      chosen = (int)v;
      loc.from_cache = 1;
    }
  }
  if (chosen == 0) {
    // exploration: real solves of the first blocks at each candidate width
    const int cands[3] = {8, 16, 32};
    double best_ms = 0.0;
    for (int w : cands) {
      if (w > maxw || done + w > m_rhs || loc.n_candidates >= 8) continue;
      blockcg_status rc = blockcg_tune(h, w);
      if (rc) return rc;
      double ms = 0.0;
      rc = solve_block(w, &ms);
      if (rc) {
        result = rc;
        break;
      }
      loc.cand_width[loc.n_candidates] = w;
      loc.cand_ms_per_rhs[loc.n_candidates] = ms / w;
      ++loc.n_candidates;
      if (chosen == 0 || ms / w < best_ms) {
        best_ms = ms / w;
        chosen = w;
      }
    }
    if (!result && chosen == 0) chosen = m_rhs < maxw ? m_rhs : maxw;  // fewer than 8 RHS
    if (!result && loc.n_candidates >= 2) cache_put(h, wkey, chosen);
  }
  while (!result && done < m_rhs) {
    const int n = (m_rhs - done) < chosen ? (m_rhs - done) : chosen;
    result = solve_block(n, nullptr);
  }
  loc.width = chosen;
  if (st) *st = loc;
  return result;
}

blockcg_status blockcg_tune(blockcg_t h, int n_rhs) {
  blockcg_status rc = check_ready(h, n_rhs);
  if (rc) return rc;
  const int N = n_rhs;
  Ws w = carve(h, N, h->ws);
  const size_t nel = (size_t)h->g.Vh * N * 3;
  CK(cudaMemsetAsync(w.P, 0, nel * elem_bytes(h->sloppy), h->stream));
  CK(cudaMemsetAsync(w.Y, 0, nel * elem_bytes(h->fine), h->stream));
  tune_block(h, w, N);
  CK(cudaStreamSynchronize(h->stream));
  return BLOCKCG_OK;
}

blockcg_status blockcg_bench_dslash(blockcg_t h, int n_rhs, int fine, int reps,
                                    double* ms_per_launch) {
  blockcg_status rc = check_ready(h, n_rhs);
  if (rc) return rc;
  if (reps < 1 || !ms_per_launch) return fail(h, BLOCKCG_ERR_ARG, "bad argument");
  const int N = n_rhs;
  Ws w = carve(h, N, h->ws);
  cudaStream_t s = h->stream;
  FieldKind k = fine ? h->fine : h->sloppy;
  const void* links = fine ? h->links_fine : h->links_sloppy;
  void* in = fine ? w.Y : w.P;
  void* out = fine ? w.Tf : w.Ts;
  size_t nel = (size_t)h->g.Vh * N * 3;
  CK(cudaMemsetAsync(in, 0, nel * elem_bytes(k), s));
  Gate g0{nullptr, GATE_ALWAYS};
  int R = stencil_R(h, k, N, links, in, out);
  // one untimed launch, then the timed ones
  KL(dslash(k, R, EPI_NONE, links, in, out, nullptr, nullptr, 0.0, h->g, 1, N, g0, s));
  EventPair ev;
  CK(ev.create());
  CK(cudaEventRecord(ev.a, s));
  for (int i = 0; i < reps; ++i)
    KL(dslash(k, R, EPI_NONE, links, in, out, nullptr, nullptr, 0.0, h->g, 1, N, g0, s));
  CK(cudaEventRecord(ev.b, s));
  CK(cudaEventSynchronize(ev.b));
  float ms = 0;
  cudaEventElapsedTime(&ms, ev.a, ev.b);
  *ms_per_launch = ms / reps;
  return BLOCKCG_OK;
}

}  // extern "C"

// ---------------------------------------------------------------------------
// Batched solves.  Each problem keeps its own handle (lattice, mass, links,
// workspace, status word) and a stream of the batch.  With graphs, the whole
// iteration loop runs on the device: one CUDA graph holds, per problem, a
// WHILE node whose body is a short chunk of gated iterations followed by a
// one-thread kernel that sets the loop condition from the problem's status
// word (not converged, no error, iteration budget left).  All WHILE nodes are
// roots, so the problems run side by side, and one graph launch solves the
// whole batch with no host round trips; the graph is built once per
// configuration (block widths, tolerance, buffers) and reused.  Without
// graphs, the host enqueues chunks on the problems' streams and polls.

struct blockcg_batch {
  std::vector<blockcg_ctx*> probs;
  cudaStream_t user;    // the caller's stream: the batch starts and ends in its order
  cudaStream_t origin;  // the batch's own stream (capture is not possible on a legacy stream)
  std::vector<cudaStream_t> streams;
  std::vector<cudaEvent_t> done_ev;
  cudaEvent_t fork_ev;
  SolverStatus* host_st;  // pinned, one per problem
  cudaGraph_t graph;
  cudaGraphExec_t exec;
  std::string graph_key;                  // configuration the graph was built for
  size_t graph_nodes;                     // kernels in all loop bodies
  std::vector<long long> graph_launches;  // kernel launches of one loop trip (or chunk), per problem
  std::map<std::string, int> tuned;       // stencil tuning shared across problems
  std::string err;
};

namespace {

blockcg_status bfail(blockcg_batch* b, blockcg_status s, const std::string& msg) {
  b->err = msg;
  return s;
}

#define BK(call)                                                                             \
  do {                                                                                       \
    cudaError_t e_ = (call);                                                                 \
    if (e_ != cudaSuccess)                                                                   \
      return bfail(b, BLOCKCG_ERR_CUDA, std::string(#call) + ": " + cudaGetErrorString(e_)); \
  } while (0)

// a problem's error, with the problem's index
blockcg_status pfail(blockcg_batch* b, int p, blockcg_status rc) {
  return bfail(b, rc, "problem " + std::to_string(p) + ": " + b->probs[p]->err);
}

void drop_graph(blockcg_batch* b) {
  if (b->exec) cudaGraphExecDestroy(b->exec);
  if (b->graph) cudaGraphDestroy(b->graph);
  b->exec = nullptr;
  b->graph = nullptr;
  b->graph_key.clear();
}

std::string tune_key(const blockcg_ctx* h, FieldKind k, int N) {
  char buf[96];
  snprintf(buf, sizeof(buf), "%d.%d.%d.%d/%d/%d", h->dims[0], h->dims[1], h->dims[2], h->dims[3],
           (int)k, N);
  return buf;
}

// stencil tuning of one problem, reusing the result of any earlier problem
// with the same lattice, storage kind and N
void batch_tune(blockcg_batch* b, blockcg_ctx* h, const Ws& w, int N) {
  const FieldKind kinds[2] = {h->sloppy, h->fine};
  if (!h->p.dslash_variant)
    for (FieldKind k : kinds) {
      auto it = b->tuned.find(tune_key(h, k, N));
      if (it != b->tuned.end()) h->tuned_R[(int)k * 128 + N] = it->second;
    }
  tune_block(h, w, N);
  if (!h->p.dslash_variant)
    for (FieldKind k : kinds) b->tuned[tune_key(h, k, N)] = h->tuned_R[(int)k * 128 + N];
}

// one chunk of iterations of every active problem, each on its stream,
// followed by the copy of its status word and the join into the origin
// stream; returns the first problem error
blockcg_status enqueue_chunk(blockcg_batch* b, const std::vector<char>& active,
                             const std::vector<int>& N, int chunk, double tol) {
  const int n = (int)b->probs.size();
  BK(cudaEventRecord(b->fork_ev, b->origin));
  for (int p = 0; p < n; ++p) {
    if (!active[p]) continue;
    blockcg_ctx* h = b->probs[p];
    Ws w = carve(h, N[p], h->ws);
    BK(cudaStreamWaitEvent(b->streams[p], b->fork_ev, 0));
    long long l0 = h->launches;
    for (int i = 0; i < chunk; ++i) {
      blockcg_status rc = iterate_block(h, w, N[p], tol);
      if (rc) return pfail(b, p, rc);
    }
    b->graph_launches[p] = h->launches - l0;
    BK(cudaMemcpyAsync(&b->host_st[p], w.st, sizeof(SolverStatus), cudaMemcpyDeviceToHost,
                       b->streams[p]));
    BK(cudaEventRecord(b->done_ev[p], b->streams[p]));
    BK(cudaStreamWaitEvent(b->origin, b->done_ev[p], 0));
  }
  return BLOCKCG_OK;
}

// iterations per loop trip of a problem in the device-looped graph: the
// caller's choice (flags bits 8..15), else min(check_every, 4)
int loop_chunk(const blockcg_ctx* h, int N, int flags) {
  const int req = (flags >> 8) & 0xff;
  if (req > 0) return req;
  int c = default_check_every(h, N);
  return c < 4 ? c : 4;
}

std::string graph_key_of(const blockcg_batch* b, const std::vector<int>& N, double tol, int flags) {
  std::string k;
  char buf[160];
  snprintf(buf, sizeof(buf), "%.17g|%d|", tol, flags);
  k += buf;
  for (size_t p = 0; p < b->probs.size(); ++p) {
    const blockcg_ctx* h = b->probs[p];
    snprintf(buf, sizeof(buf), "%d,%p,%p,%d,%d,%g,%d;", N[p], (const void*)h->ws, h->gauge,
             h->p.max_iter, h->p.ru_every, h->p.ru_delta, h->p.dslash_variant);
    k += buf;
  }
  return k;
}

// one graph, one WHILE node per problem; each body = loop_chunk gated
// iterations + the loop-condition kernel
blockcg_status build_loop_graph(blockcg_batch* b, const std::vector<int>& N, double tol,
                                int flags) {
  drop_graph(b);
  BK(cudaGraphCreate(&b->graph, 0));
  size_t kernels = 0;
  for (size_t p = 0; p < b->probs.size(); ++p) {
    blockcg_ctx* h = b->probs[p];
    Ws w = carve(h, N[p], h->ws);
    const int chunk = loop_chunk(h, N[p], flags);
    const int max_trips = (h->p.max_iter + chunk - 1) / chunk + 2;
    cudaGraphConditionalHandle hnd;
    BK(cudaGraphConditionalHandleCreate(&hnd, b->graph, 1, cudaGraphCondAssignDefault));
    // zeroed storage: the parameter union has no default constructor
    alignas(cudaGraphNodeParams) unsigned char np_raw[sizeof(cudaGraphNodeParams)];
    memset(np_raw, 0, sizeof(np_raw));
    cudaGraphNodeParams* np = reinterpret_cast<cudaGraphNodeParams*>(np_raw);
    np->type = cudaGraphNodeTypeConditional;
    np->conditional.handle = hnd;
    np->conditional.type = cudaGraphCondTypeWhile;
    np->conditional.size = 1;
    cudaGraphNode_t node;
    BK(cudaGraphAddNode(&node, b->graph, nullptr, nullptr, 0, np));
    cudaGraph_t body = np->conditional.phGraph_out[0];
    BK(cudaStreamBeginCaptureToGraph(b->streams[p], body, nullptr, nullptr, 0,
                                     cudaStreamCaptureModeRelaxed));
    const long long l0 = h->launches;
    blockcg_status rc = BLOCKCG_OK;
    for (int i = 0; i < chunk && !rc; ++i) rc = iterate_block(h, w, N[p], tol);
    cudaError_t e = cudaSuccess;
    if (!rc) {
      e = loop_condition(hnd, w.st, max_trips, b->streams[p]);
      ++h->launches;
    }
    cudaGraph_t captured = nullptr;
    cudaError_t e2 = cudaStreamEndCapture(b->streams[p], &captured);
    if (rc) {
      cudaGetLastError();
      drop_graph(b);
      return pfail(b, (int)p, rc);
    }
    if (e != cudaSuccess || e2 != cudaSuccess) {
      cudaGetLastError();
      drop_graph(b);
      return bfail(b, BLOCKCG_ERR_CUDA,
                   std::string("loop graph capture: ") +
                       cudaGetErrorString(e != cudaSuccess ? e : e2));
    }
    b->graph_launches[p] = h->launches - l0;
    kernels += (size_t)(h->launches - l0);
  }
  BK(cudaGraphInstantiate(&b->exec, b->graph, 0));
  b->graph_nodes = kernels;
  b->graph_key = graph_key_of(b, N, tol, flags);
  return BLOCKCG_OK;
}

// restores each handle's stream and profiling flag when a batch solve ends
struct BatchGuard {
  blockcg_batch* b;
  std::vector<cudaStream_t> s;
  std::vector<int> prof;
  explicit BatchGuard(blockcg_batch* bb) : b(bb) {
    for (blockcg_ctx* h : b->probs) {
      s.push_back(h->stream);
      prof.push_back(h->p.profile);
    }
    for (size_t p = 0; p < b->probs.size(); ++p) {
      b->probs[p]->stream = b->streams[p];
      b->probs[p]->p.profile = 0;
    }
  }
  ~BatchGuard() {
    for (size_t p = 0; p < b->probs.size(); ++p) {
      b->probs[p]->stream = s[p];
      b->probs[p]->p.profile = prof[p];
    }
  }
};

}  // namespace

extern "C" {

blockcg_status blockcg_batch_create(blockcg_batch_t* out, const blockcg_t* problems, int n,
                                    void* stream) {
  if (!out) return BLOCKCG_ERR_ARG;
  *out = nullptr;
  if (!problems || n < 1 || n > BLOCKCG_BATCH_MAX) return BLOCKCG_ERR_ARG;
  for (int p = 0; p < n; ++p) {
    if (!problems[p]) return BLOCKCG_ERR_ARG;
    for (int q = 0; q < p; ++q)
      if (problems[q] == problems[p]) return BLOCKCG_ERR_ARG;  // one workspace per problem
  }
  blockcg_batch* b = new blockcg_batch();
  b->user = (cudaStream_t)stream;
  b->origin = nullptr;
  b->graph = nullptr;
  b->exec = nullptr;
  b->graph_nodes = 0;
  b->host_st = nullptr;
  b->fork_ev = nullptr;
  b->probs.assign(problems, problems + n);
  b->graph_launches.assign(n, 0);
  bool ok = cudaEventCreateWithFlags(&b->fork_ev, cudaEventDisableTiming) == cudaSuccess &&
            cudaStreamCreateWithFlags(&b->origin, cudaStreamNonBlocking) == cudaSuccess &&
            cudaMallocHost((void**)&b->host_st, n * sizeof(SolverStatus)) == cudaSuccess;
  for (int p = 0; ok && p < n; ++p) {
    cudaStream_t s = nullptr;
    cudaEvent_t e = nullptr;
    ok = cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking) == cudaSuccess;
    if (ok) b->streams.push_back(s);
    ok = ok && cudaEventCreateWithFlags(&e, cudaEventDisableTiming) == cudaSuccess;
    if (ok) b->done_ev.push_back(e);
  }
  if (!ok) {
    cudaGetLastError();
    blockcg_batch_destroy(b);
    return BLOCKCG_ERR_CUDA;
  }
  memset(b->host_st, 0, n * sizeof(SolverStatus));
  *out = b;
  return BLOCKCG_OK;
}

void blockcg_batch_destroy(blockcg_batch_t b) {
  if (!b) return;
  drop_graph(b);
  for (cudaStream_t s : b->streams) {
    cudaStreamSynchronize(s);
    cudaStreamDestroy(s);
  }
  for (cudaEvent_t e : b->done_ev) cudaEventDestroy(e);
  if (b->origin) {
    cudaStreamSynchronize(b->origin);
    cudaStreamDestroy(b->origin);
  }
  if (b->fork_ev) cudaEventDestroy(b->fork_ev);
  if (b->host_st) cudaFreeHost(b->host_st);
  delete b;
}

const char* blockcg_batch_last_error(blockcg_batch_t b) { return b ? b->err.c_str() : "null batch"; }

blockcg_status blockcg_batch_solve(blockcg_batch_t b, const void* const* B, void* const* X,
                                   const int* n_rhs, double tol, int flags, blockcg_stats* stats,
                                   int* status, blockcg_batch_stats* bstats) {
  if (!b) return BLOCKCG_ERR_ARG;
  if (!B || !X || !n_rhs) return bfail(b, BLOCKCG_ERR_ARG, "null pointer");
  const int n = (int)b->probs.size();
  std::vector<int> N(n);
  for (int p = 0; p < n; ++p) {
    blockcg_status rc = check_solve_args(b->probs[p], B[p], X[p], n_rhs[p], tol);
    if (rc) return pfail(b, p, rc);
    N[p] = n_rhs[p];
  }
  const bool use_graph = (flags & BLOCKCG_BATCH_GRAPH) != 0;
  BatchGuard guard(b);
  EventPair ev;
  BK(ev.create());
  cudaEvent_t e0 = ev.a, e1 = ev.b;
  // the batch runs after the caller's earlier work on its stream
  BK(cudaEventRecord(b->fork_ev, b->user));
  BK(cudaStreamWaitEvent(b->origin, b->fork_ev, 0));
  BK(cudaEventRecord(e0, b->origin));
  BK(cudaEventRecord(b->fork_ev, b->origin));
  long long launches = 0;
  // stencil tuning first (timed launches, one problem at a time), then the
  // set-up of every problem on its own stream
  for (int p = 0; p < n; ++p) {
    blockcg_ctx* h = b->probs[p];
    reset_instrumentation(h);
    BK(cudaStreamWaitEvent(b->streams[p], b->fork_ev, 0));
    batch_tune(b, h, carve(h, N[p], h->ws), N[p]);
  }
  int chunk = 32;
  for (int p = 0; p < n; ++p) {
    blockcg_ctx* h = b->probs[p];
    Ws w = carve(h, N[p], h->ws);
    long long l0 = h->launches;
    blockcg_status rc = solve_begin(h, w, B[p], X[p], N[p], tol);
    if (rc) return pfail(b, p, rc);
    launches += h->launches - l0;
    BK(cudaEventRecord(b->done_ev[p], b->streams[p]));
    BK(cudaStreamWaitEvent(b->origin, b->done_ev[p], 0));
    int c = default_check_every(h, N[p]);
    if (c < chunk) chunk = c;
  }
  long long replays = 0, captures = 0;
  if (use_graph) {
    // the whole iteration loop of every problem in one graph launch
    if (!b->exec || b->graph_key != graph_key_of(b, N, tol, flags)) {
      blockcg_status rc = build_loop_graph(b, N, tol, flags);
      if (rc) return rc;
      ++captures;
    }
    BK(cudaGraphLaunch(b->exec, b->origin));
    ++replays;
    for (int p = 0; p < n; ++p) {
      Ws w = carve(b->probs[p], N[p], b->probs[p]->ws);
      BK(cudaMemcpyAsync(&b->host_st[p], w.st, sizeof(SolverStatus), cudaMemcpyDeviceToHost,
                         b->origin));
    }
    BK(cudaStreamSynchronize(b->origin));
    for (int p = 0; p < n; ++p) launches += b->host_st[p].trips * b->graph_launches[p];
  } else {
    // host-driven: chunks on the problems' streams, status polled between them
    std::vector<char> active(n, 1);
    std::vector<int> launched(n, 0);
    for (;;) {
      int n_active = 0;
      for (int p = 0; p < n; ++p) n_active += active[p];
      if (!n_active) break;
      blockcg_status rc = enqueue_chunk(b, active, N, chunk, tol);
      if (rc) return rc;
      BK(cudaStreamSynchronize(b->origin));
      for (int p = 0; p < n; ++p) {
        if (!active[p]) continue;
        launches += b->graph_launches[p];
        launched[p] += chunk;
        const SolverStatus& hs = b->host_st[p];
        if (hs.done || hs.error || hs.iters >= b->probs[p]->p.max_iter ||
            launched[p] >= b->probs[p]->p.max_iter)
          active[p] = 0;
      }
    }
  }
  // native-FP64 confirmation of every convergence a double-float reliable
  // update reported: enqueued for all such problems, then one wait
  bool verifying = false;
  for (int p = 0; p < n; ++p) {
    blockcg_ctx* h = b->probs[p];
    const SolverStatus& hs = b->host_st[p];
    if (hs.error || !hs.done || converged(h, hs)) continue;
    Ws w = carve(h, N[p], h->ws);
    long long l0 = h->launches;
    blockcg_status rc = verify_fp64(h, w, N[p], tol);
    if (rc) return pfail(b, p, rc);
    launches += h->launches - l0;
    BK(cudaMemcpyAsync(&b->host_st[p], w.st, sizeof(SolverStatus), cudaMemcpyDeviceToHost,
                       b->streams[p]));
    verifying = true;
  }
  if (verifying)
    for (int p = 0; p < n; ++p) BK(cudaStreamSynchronize(b->streams[p]));
  // results: a failed confirmation continues on the host (rare), max_iter
  // handling and the copy-out, each problem on its stream
  blockcg_status first = BLOCKCG_OK;
  for (int p = 0; p < n; ++p) {
    blockcg_ctx* h = b->probs[p];
    Ws w = carve(h, N[p], h->ws);
    SolverStatus hs = b->host_st[p];
    blockcg_status result = BLOCKCG_OK;
    long long l0 = h->launches;
    if (!hs.error && !converged(h, hs) && hs.iters < h->p.max_iter && !hs.stopped) {
      blockcg_status rc = host_loop(h, w, N[p], tol, &hs);
      if (rc) return pfail(b, p, rc);
    }
    blockcg_status rc = solve_end(h, w, X[p], N[p], tol, &hs, &result);
    if (rc) return pfail(b, p, rc);
    launches += h->launches - l0;
    if (status) status[p] = result;
    if (result && !first) {
      first = result;
      b->err = "problem " + std::to_string(p) + ": " + h->err;
    }
    if (stats) {
      double* per_rhs = stats[p].true_rel_res;  // the caller's array (or NULL)
      memset(&stats[p], 0, sizeof(blockcg_stats));
      stats[p].true_rel_res = per_rhs;
      stats[p].iters = hs.iters;
      stats[p].reliable_updates = hs.reliable_updates;
      stats[p].true_rel_res_max = hs.true_res_max;
      if (per_rhs)
        BK(cudaMemcpyAsync(per_rhs, w.tres, N[p] * sizeof(double), cudaMemcpyDeviceToHost,
                           b->streams[p]));
    }
    BK(cudaEventRecord(b->done_ev[p], b->streams[p]));
    BK(cudaStreamWaitEvent(b->origin, b->done_ev[p], 0));
  }
  BK(cudaEventRecord(e1, b->origin));
  BK(cudaStreamWaitEvent(b->user, e1, 0));
  BK(cudaEventSynchronize(e1));
  float ms = 0;
  cudaEventElapsedTime(&ms, e0, e1);
  if (stats)
    for (int p = 0; p < n; ++p) stats[p].ms_total = ms;
  if (bstats) {
    bstats->ms_total = ms;
    bstats->chunk = use_graph ? loop_chunk(b->probs[0], N[0], flags) : chunk;
    bstats->graph_replays = replays;
    bstats->graph_captures = captures;
    bstats->graph_nodes = (long long)b->graph_nodes;
    bstats->launches = launches;
  }
  return first;
}

}  // extern "C"
