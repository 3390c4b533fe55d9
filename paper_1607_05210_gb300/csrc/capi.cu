// C ABI (include/hapod.h): context, rooted tree, tolerance split and the batch
// scheduler that runs every ready node of the tree together.
//
// Tree and tolerances (Sec. 3.1 Def. Rooted Tree, Sec. 3.3 Thm.
// cor:hapod_bound) are host FP64 arithmetic done once in hapod_create.  A node is
// ready once all of its inputs exist (Def. HAPOD: leaf input D^-1(a), inner input
// the union of the children's sigma-scaled modes).  All ready nodes run as one
// batch: one grouped launch per step (Gram, eigensolve, truncation, gather,
// modes), one host read-back of the kept ranks per batch.  A child writes its
// modes straight into its parent's input buffer when every sibling finishes in the
// same batch (balanced trees); otherwise it parks them in its own buffer until
// the parent's buffer can be sized exactly.  Device memory comes from a
// stream-ordered pool; a node's owned input is freed as soon as its modes exist
// (Sec. 3.4, reduced memory requirements).
#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <map>
#include <mutex>
#include <tuple>
#include <new>
#include <string>
#include <vector>

#include "hapod_internal.cuh"

using namespace hapod;

namespace {

thread_local std::string g_thread_error = "no error";

// ------------------------------------------------------------------ memory pool
std::mutex g_pool_mu;
std::vector<cudaMemPool_t> g_pools;

cudaError_t get_pool(int dev, cudaMemPool_t* out) {
  std::lock_guard<std::mutex> lk(g_pool_mu);
  if ((int)g_pools.size() <= dev) g_pools.resize(dev + 1, nullptr);
  if (!g_pools[dev]) {
    cudaMemPoolProps props;
    memset(&props, 0, sizeof(props));
    props.allocType = cudaMemAllocationTypePinned;
    props.location.type = cudaMemLocationTypeDevice;
    props.location.id = dev;
    cudaMemPool_t p;
    cudaError_t e = cudaMemPoolCreate(&p, &props);
    if (e != cudaSuccess) return e;
    uint64_t thr = UINT64_MAX;
    cudaMemPoolSetAttribute(p, cudaMemPoolAttrReleaseThreshold, &thr);
    g_pools[dev] = p;
  }
  *out = g_pools[dev];
  return cudaSuccess;
}

// Per-step CUDA-event accounting (HAPOD_FLAG_PROFILE).
struct Prof {
  struct Rec {
    int step;
    cudaEvent_t a, b;
  };
  std::vector<Rec> pending;
  std::vector<cudaEvent_t> spare;
  hapod_profile_info acc;
  Prof() { memset(&acc, 0, sizeof(acc)); }
  cudaEvent_t get() {
    if (!spare.empty()) {
      cudaEvent_t e = spare.back();
      spare.pop_back();
      return e;
    }
    cudaEvent_t e = nullptr;
    cudaEventCreate(&e);
    return e;
  }
  // call after the stream has been synchronised
  void resolve() {
    for (Rec& r : pending) {
      float ms = 0.f;
      if (cudaEventElapsedTime(&ms, r.a, r.b) == cudaSuccess) acc.ms[r.step] += ms;
      spare.push_back(r.a);
      spare.push_back(r.b);
    }
    pending.clear();
    cudaGetLastError();
  }
  ~Prof() {
    for (Rec& r : pending) {
      cudaEventDestroy(r.a);
      cudaEventDestroy(r.b);
    }
    for (cudaEvent_t e : spare) cudaEventDestroy(e);
  }
};

struct Env {
  Prof* prof = nullptr;
  HostStage* stage = nullptr;  // contexts: staged uploads (see HostStage)
  int* err_dev = nullptr;  // bounded-wait error flag of the tensor-core kernels (per batch)
  int dev = 0;
  cudaStream_t s = nullptr;
  cudaMemPool_t pool = nullptr;
  std::string err;
  hapod_status code = HAPOD_OK;

  bool fail(hapod_status c, const std::string& msg) {
    if (code == HAPOD_OK || code >= HAPOD_WARN_NOCONVERGE) {
      code = c;
      err = msg;
    }
    return false;
  }
  bool cuda(cudaError_t e, const char* what) {
    if (e == cudaSuccess) return true;
    cudaGetLastError();
    return fail(e == cudaErrorMemoryAllocation ? HAPOD_ERR_OOM : HAPOD_ERR_CUDA,
                std::string(what) + ": " + cudaGetErrorString(e));
  }
  void* alloc(size_t bytes, const char* what) {
    if (bytes == 0) bytes = 16;
    void* p = nullptr;
    cudaError_t e = cudaMallocFromPoolAsync(&p, bytes, pool, s);
    if (e != cudaSuccess) {
      cuda(e, what);
      return nullptr;
    }
    return p;
  }
  void release(void* p) {
    if (p) cudaFreeAsync(p, s);
  }
  // profiling brackets around a step's launches (no-ops without a profiler)
  cudaEvent_t tic() {
    if (!prof) return nullptr;
    cudaEvent_t e = prof->get();
    if (e) cudaEventRecord(e, s);
    return e;
  }
  void toc(cudaEvent_t a, int step, int launches, double bytes, double flops) {
    if (!prof || !a) return;
    cudaEvent_t b = prof->get();
    if (!b) return;
    cudaEventRecord(b, s);
    prof->pending.push_back({step, a, b});
    prof->acc.launches[step] += launches;
    prof->acc.bytes[step] += bytes;
    prof->acc.flops[step] += flops;
  }
  template <typename T>
  T* upload(const std::vector<T>& v, const char* what) {
    T* d = static_cast<T*>(alloc(sizeof(T) * std::max<size_t>(1, v.size()), what));
    if (!d) return nullptr;
    if (!v.empty() && !cuda(staged_upload(stage, d, v.data(), sizeof(T) * v.size(), s), what)) {
      release(d);
      return nullptr;
    }
    return d;
  }
};

// Debug only: HAPOD_DEBUG_WAIT_CYCLES=N (N > 0) shortens every bounded device-side
// wait of the tensor-core kernels to N clock cycles, so that a test can make one run
// out on a healthy kernel; unset, the budget is about one second.  The value is read at
// every call and stored in err[1] of the kernels' error flag.
int debug_wait_cycles() {
  const char* e = getenv("HAPOD_DEBUG_WAIT_CYCLES");
  if (!e || !*e) return 0;
  const long long v = atoll(e);
  return v > 0 ? (int)std::min<long long>(v, 1 << 30) : 0;
}

// err[0] = 0 and err[1] = 0 are set by the caller's memset; this stores the debug budget.
bool init_err_flag(Env& env, int* err) {
  static thread_local int budget = 0;  // staged by the copy before it returns (pageable source)
  budget = debug_wait_cycles();
  if (budget <= 0) return true;
  return env.cuda(cudaMemcpyAsync(err + 1, &budget, sizeof(int), cudaMemcpyHostToDevice, env.s), "set wait budget");
}

__global__ void staged_copy_kernel(uint4* __restrict__ dst, const uint4* __restrict__ src, size_t n16,
                                   uint8_t* __restrict__ dtail, const uint8_t* __restrict__ stail, int ntail) {
  for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < n16; i += (size_t)gridDim.x * blockDim.x)
    dst[i] = src[i];
  if (blockIdx.x == 0 && (int)threadIdx.x < ntail) dtail[threadIdx.x] = stail[threadIdx.x];
}

}  // namespace

cudaError_t hapod::staged_upload(HostStage* st, void* dst, const void* src, size_t bytes, cudaStream_t s) {
  if (bytes == 0) return cudaSuccess;
  if (!st || !st->base || bytes > st->cap || (reinterpret_cast<uintptr_t>(dst) & 15))
    return cudaMemcpyAsync(dst, src, bytes, cudaMemcpyHostToDevice, s);
  if (st->used + bytes > st->cap) {  // every earlier copy kernel has read its bytes once s is idle
    const cudaError_t e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) return e;
    st->used = 0;
  }
  uint8_t* h = st->base + st->used;
  memcpy(h, src, bytes);
  st->used += (bytes + 15) & ~size_t(15);
  const size_t n16 = bytes / 16;
  const unsigned blocks = (unsigned)std::min<size_t>(64, n16 / 256 + 1);
  staged_copy_kernel<<<blocks, 256, 0, s>>>(static_cast<uint4*>(dst), reinterpret_cast<const uint4*>(h), n16,
                                            static_cast<uint8_t*>(dst) + n16 * 16, h + n16 * 16, (int)(bytes % 16));
  return cudaGetLastError();
}

namespace {

bool init_env(Env& env, void* stream) {
  env.s = static_cast<cudaStream_t>(stream);
  if (!env.cuda(cudaGetDevice(&env.dev), "cudaGetDevice")) return false;
  return env.cuda(get_pool(env.dev, &env.pool), "memory pool");
}

bool valid_precision(int p) {
  return p == HAPOD_FP64 || p == HAPOD_MIXED_TF32X3 || p == HAPOD_FP64_OZAKI || p == HAPOD_MIXED_BF16X3 ||
         p == HAPOD_MIXED_FX3;
}
// FP64 snapshots (the FP64 and digit-slice forms) versus FP32 snapshots (mixed forms)
bool f64_data(int p) { return p == HAPOD_FP64 || p == HAPOD_FP64_OZAKI; }
bool mixed_form(int p) { return p == HAPOD_MIXED_TF32X3 || p == HAPOD_MIXED_BF16X3 || p == HAPOD_MIXED_FX3; }
size_t elem_size(int p) { return f64_data(p) ? sizeof(double) : sizeof(float); }

// ------------------------------------------------------------- batched steps
// One node of a batch: its input and the per-node device buffers of the steps.
struct Work {
  const void* X = nullptr;
  int64_t ldx = 0;
  void* X_tmp = nullptr;  // 16-byte aligned copy for TMA when the input is not
  int64_t n = 0;
  int64_t m = 0;
  double eps = 0.0;
  // device buffers
  double* G = nullptr;
  void* A = nullptr;
  void* V = nullptr;
  double* lam_tmp = nullptr;
  double* lambda = nullptr;
  int32_t* perm = nullptr;
  double* sigma = nullptr;
  double* Vk = nullptr;
  // results
  NodeResult res{};
  std::vector<double> sigma_host;
  // modes destination
  void* Y = nullptr;
  int64_t ldy = 0;
  double* scale = nullptr;  // device 1/sigma (root)
  int32_t* exps = nullptr;  // digit-slice form: column exponents (owned)
  int64_t ldvk = 0;         // leading dimension of Vk (0: m)
};

constexpr int kMaxSweeps = 40;

bool alloc_work(Env& env, std::vector<Work*>& ws, bool fp64) {
  const size_t t = fp64 ? sizeof(double) : sizeof(float);
  for (Work* w : ws) {
    const size_t mm = (size_t)w->m * w->m;
    w->G = (double*)env.alloc(mm * sizeof(double), "alloc G");
    w->A = env.alloc(mm * sizeof(double), "alloc Cholesky factor");
    w->V = env.alloc(mm * t, "alloc eigenvectors");
    w->lam_tmp = (double*)env.alloc(w->m * sizeof(double), "alloc lambda");
    w->lambda = (double*)env.alloc(w->m * sizeof(double), "alloc lambda");
    w->perm = (int32_t*)env.alloc(w->m * sizeof(int32_t), "alloc perm");
    w->sigma = (double*)env.alloc(w->m * sizeof(double), "alloc sigma");
    if (!w->G || !w->A || !w->V || !w->lam_tmp || !w->lambda || !w->perm || !w->sigma) return false;
  }
  return true;
}

void free_work(Env& env, std::vector<Work*>& ws) {
  for (Work* w : ws) {
    env.release(w->G);
    env.release(w->A);
    env.release(w->V);
    env.release(w->lam_tmp);
    env.release(w->lambda);
    env.release(w->perm);
    env.release(w->sigma);
    env.release(w->Vk);
    env.release(w->X_tmp);
    env.release(w->exps);
    w->exps = nullptr;
    w->X_tmp = nullptr;
    w->G = nullptr;
    w->A = w->V = nullptr;
    w->lam_tmp = w->lambda = w->sigma = w->Vk = nullptr;
    w->perm = nullptr;
  }
}

// ------------------------------------------------------------- digit-slice form
// The digit planes of a node's X (14 bytes per element) are produced in rounds of at
// most oz_digit_cap() bytes; a node taller than that is cut into row chunks.  The
// cap defaults to 4 GiB; the environment variable HAPOD_OZ_WORKSPACE_MB overrides it
// (read at every call).
size_t oz_digit_cap() {
  const char* e = getenv("HAPOD_OZ_WORKSPACE_MB");
  if (e && *e) {
    const long long mb = atoll(e);
    if (mb > 0) return (size_t)mb << 20;
  }
  return (size_t)4 << 30;
}

struct OzChunk {
  int node;
  int64_t r0, rows;
  int32_t CGs, RG;
  size_t bytes;
  int32_t splits, sps;  // Gram: row splits and 16-row stages per split
  int64_t slot0;        // Gram: first partial slot of the chunk within its node
};

// Row chunks of every node and rounds of consecutive chunks within the cap.
void oz_plan(const std::vector<Work*>& ws, std::vector<OzChunk>& chunks, std::vector<std::pair<size_t, size_t>>& rounds,
             size_t& max_round) {
  const size_t cap = oz_digit_cap();
  for (int i = 0; i < (int)ws.size(); ++i) {
    const int32_t CGs = oz_stored_groups(ws[i]->m);
    const size_t row_bytes = (size_t)CGs * 8 * kOzDigits * 2;
    int64_t R = (int64_t)(cap / row_bytes) / kOzKBlock * kOzKBlock;
    R = std::max<int64_t>(R, kOzKBlock);
    for (int64_t r0 = 0; r0 < ws[i]->n; r0 += R) {
      OzChunk c;
      c.node = i;
      c.r0 = r0;
      c.rows = std::min(R, ws[i]->n - r0);
      c.CGs = CGs;
      c.RG = (int32_t)oz_row_groups(c.rows);
      c.bytes = (size_t)c.RG * 8 * row_bytes;
      c.splits = c.sps = 0;
      c.slot0 = 0;
      chunks.push_back(c);
    }
  }
  max_round = 0;
  for (size_t a = 0; a < chunks.size();) {
    size_t b = a, bytes = 0;
    while (b < chunks.size() && (b == a || bytes + chunks[b].bytes <= cap)) bytes += chunks[b++].bytes;
    rounds.push_back({a, b});
    max_round = std::max(max_round, bytes + kOzDigitSlack);
    a = b;
  }
}

OzSplitJob oz_split_job(const Work* w, const OzChunk& C, uint16_t* dblk, int64_t block_base) {
  OzSplitJob S;
  memset(&S, 0, sizeof(S));
  S.X = static_cast<const double*>(w->X);
  S.ldx = w->ldx;
  S.r0 = C.r0;
  S.rows = C.rows;
  S.exps = w->exps;
  S.digits = dblk;
  S.block_base = block_base;
  S.m = (int32_t)w->m;
  S.CGs = C.CGs;
  return S;
}

// Column exponents E_j of every node without them (w->exps, owned by the Work).
bool oz_exponents(Env& env, std::vector<Work*>& ws) {
  std::vector<OzColJob> cj;
  int64_t total = 0;
  for (Work* w : ws) {
    if (w->exps) continue;
    w->exps = (int32_t*)env.alloc(sizeof(int32_t) * std::max<int64_t>(1, w->m), "alloc exponents");
    if (!w->exps) return false;
    OzColJob J;
    memset(&J, 0, sizeof(J));
    J.X = static_cast<const double*>(w->X);
    J.ldx = w->ldx;
    J.n = w->n;
    J.exps = w->exps;
    J.col_base = total;
    J.m = (int32_t)w->m;
    total += w->m;
    cj.push_back(J);
  }
  if (cj.empty()) return true;
  OzColJob* d = env.upload(cj, "upload exponent jobs");
  bool ok = d && env.cuda(launch_oz_colmax(d, (int)cj.size(), total, env.s), "exponent launch");
  env.release(d);
  return ok;
}

// K1, digit-slice FP64 form: exponents, then per round the digit planes and the
// tensor-core Gram tiles of its chunks, then one reduce of the split partials.
constexpr int kStepDigits = 6;  // profile index of the digit conversion (include/hapod.h)

bool step_gram_oz(Env& env, std::vector<Work*>& ws) {
  if (ws.empty()) return true;
  const int nw = (int)ws.size();
  double bytes = 0, flops = 0, dbytes = 0;
  for (Work* w : ws) {
    bytes += 8.0 * w->n * w->m;
    flops += (double)w->n * w->m * (w->m + 1);
    dbytes += 22.0 * w->n * w->m;
  }
  cudaEvent_t t0 = env.tic();
  if (!oz_exponents(env, ws)) return false;
  env.toc(t0, kStepDigits, 1, 0.0, 0.0);
  std::vector<OzChunk> chunks;
  std::vector<std::pair<size_t, size_t>> rounds;
  size_t max_round = 0;
  oz_plan(ws, chunks, rounds, max_round);
  std::vector<int64_t> node_slots(nw, 0);
  for (const auto& rd : rounds) {
    // splits: about two waves of one CTA per SM over the round's tiles, whole 256-row blocks
    int64_t T = 0;
    for (size_t c = rd.first; c < rd.second; ++c) T += oz_gram_tiles((int32_t)ws[chunks[c].node]->m);
    const int64_t want = std::max<int64_t>(1, (2 * kNumSMs) / std::max<int64_t>(1, T));
    for (size_t c = rd.first; c < rd.second; ++c) {
      OzChunk& C = chunks[c];
      const int64_t stages = C.RG / 2;
      const int64_t blk = kOzKBlock / 16;
      int64_t sps = (stages + want - 1) / want;
      sps = std::max<int64_t>(blk, (sps + blk - 1) / blk * blk);
      sps = std::min<int64_t>(sps, (int64_t)1 << 18);  // int64 flush sums stay exact (<= 2^22 rows)
      C.sps = (int32_t)sps;
      C.splits = (int32_t)((stages + sps - 1) / sps);
      C.slot0 = node_slots[C.node];
      node_slots[C.node] += C.splits;
    }
  }
  std::vector<int64_t> node_base(nw, 0);
  size_t total_partial = 0;
  for (int i = 0; i < nw; ++i) {
    const int64_t mp = ws[i]->m;
    node_base[i] = (int64_t)total_partial;
    total_partial += (size_t)node_slots[i] * mp * mp;
  }
  double* partial = (double*)env.alloc(sizeof(double) * std::max<size_t>(1, total_partial), "alloc gram partials");
  uint16_t* digits = (uint16_t*)env.alloc(std::max<size_t>(16, max_round), "alloc digit planes");
  bool ok = partial && digits;
  std::vector<void*> job_bufs;
  for (size_t r = 0; r < rounds.size() && ok; ++r) {
    std::vector<OzSplitJob> sj;
    std::vector<OzGramJob> gj;
    std::vector<CUtensorMap> gm;
    size_t off = 0;
    int64_t blocks = 0, items = 0;
    for (size_t c = rounds[r].first; c < rounds[r].second; ++c) {
      const OzChunk& C = chunks[c];
      Work* w = ws[C.node];
      uint16_t* dblk = reinterpret_cast<uint16_t*>(reinterpret_cast<uint8_t*>(digits) + off);
      off += C.bytes;
      sj.push_back(oz_split_job(w, C, dblk, blocks));
      blocks += oz_split_blocks(C.rows, C.CGs);
      OzGramJob G;
      memset(&G, 0, sizeof(G));
      const int64_t mp = w->m;
      G.digits = dblk;
      G.exps = w->exps;
      G.partial = partial + node_base[C.node] + (size_t)C.slot0 * mp * mp;
      G.item_base = items;
      G.RG = C.RG;
      G.CGs = C.CGs;
      G.m = (int32_t)w->m;
      G.mp = (int32_t)mp;
      G.splits = C.splits;
      G.stages_per_split = C.sps;
      G.tiles = oz_gram_tiles((int32_t)w->m);
      items += (int64_t)C.splits * G.tiles;
      gj.push_back(G);
      CUtensorMap ma, mb;
      if (!encode_oz_digits(&ma, dblk, C.CGs, C.RG, kOzGramAGroups) ||
          !encode_oz_digits(&mb, dblk, C.CGs, C.RG, kOzGramBGroups)) {
        ok = false;
        env.fail(HAPOD_ERR_CUDA, "digit tensor map: cuTensorMapEncodeTiled failed");
        break;
      }
      gm.push_back(ma);
      gm.push_back(mb);
    }
    if (!ok) break;
    OzSplitJob* sj_d = env.upload(sj, "upload split jobs");
    OzGramJob* gj_d = env.upload(gj, "upload gram jobs");
    CUtensorMap* gm_d = env.upload(gm, "upload digit tensor maps");
    job_bufs.push_back(sj_d);
    job_bufs.push_back(gj_d);
    job_bufs.push_back(gm_d);
    cudaEvent_t ts = env.tic();
    ok = sj_d && gj_d && gm_d && env.cuda(launch_oz_split(sj_d, (int)sj.size(), blocks, env.s), "digit split launch");
    env.toc(ts, kStepDigits, 1, r == 0 ? dbytes : 0.0, 0.0);
    cudaEvent_t tg = env.tic();
    ok = ok && env.cuda(launch_gram_oz(gj_d, gm_d, (int)gj.size(), items, env.err_dev, env.s), "gram launch");
    env.toc(tg, 0, 1, r == 0 ? bytes : 0.0, r == 0 ? flops : 0.0);
  }
  if (ok) {
    std::vector<OzReduceJob> rj(nw);
    int64_t cols = 0;
    for (int i = 0; i < nw; ++i) {
      memset(&rj[i], 0, sizeof(OzReduceJob));
      rj[i].partial = partial + node_base[i];
      rj[i].G = ws[i]->G;
      rj[i].col_base = cols;
      rj[i].slots = (int32_t)node_slots[i];
      rj[i].m = (int32_t)ws[i]->m;
      rj[i].mp = (int32_t)ws[i]->m;
      cols += ws[i]->m;
    }
    OzReduceJob* rj_d = env.upload(rj, "upload reduce jobs");
    job_bufs.push_back(rj_d);
    cudaEvent_t tr = env.tic();
    ok = rj_d && env.cuda(launch_oz_reduce(rj_d, nw, cols, env.s), "gram reduce launch");
    env.toc(tr, 0, 1, 0.0, 0.0);
  }
  for (void* p : job_bufs) env.release(p);
  env.release(partial);
  env.release(digits);
  return ok;
}

// K4, digit-slice FP64 form: Y = X V_k (diag scale) for every w (k = w->res.k > 0,
// V_k in w->Vk): digits of V_k, then one persistent tensor-core launch that converts
// X to digits on the fly.  Exponents are the Gram's (or computed here).
bool step_modes_oz(Env& env, std::vector<Work*>& ws) {
  if (ws.empty()) return true;
  const int nw = (int)ws.size();
  if (!oz_exponents(env, ws)) return false;
  const int NT = oz_modes_tile(0);
  std::vector<OzVSplitJob> vj(nw);
  std::vector<OzModesJob> mj(nw);
  std::vector<void*> bufs;
  int64_t vcols = 0, items = 0;
  bool ok = true;
  for (int i = 0; i < nw && ok; ++i) {
    Work* w = ws[i];
    const int32_t CGp = oz_col_groups(w->m);
    const int32_t n_tiles = (w->res.k + NT - 1) / NT;
    const int32_t NG = n_tiles * NT / 8;
    uint16_t* vdig = (uint16_t*)env.alloc((size_t)CGp * NG * kOzGroupBytes, "alloc V digits");
    int32_t* fexp = (int32_t*)env.alloc(sizeof(int32_t) * NG * 8, "alloc mode exponents");
    bufs.push_back(vdig);
    bufs.push_back(fexp);
    ok = vdig && fexp;
    OzVSplitJob& J = vj[i];
    memset(&J, 0, sizeof(J));
    J.V = w->Vk;
    J.ldv = w->ldvk ? w->ldvk : w->m;
    J.exps = w->exps;
    J.vdig = vdig;
    J.fexp = fexp;
    J.col_base = vcols;
    J.m = (int32_t)w->m;
    J.k = w->res.k;
    J.NG = NG;
    J.CGp = CGp;
    vcols += (int64_t)NG * 8;
    OzModesJob& M = mj[i];
    memset(&M, 0, sizeof(M));
    M.X = static_cast<const double*>(w->X);
    M.ldx = w->ldx;
    M.exps = w->exps;
    M.vdig = vdig;
    M.fexp = fexp;
    M.scale = w->scale;
    M.Y = static_cast<double*>(w->Y);
    M.ldy = w->ldy;
    M.n = w->n;
    M.item_base = items;
    M.m = (int32_t)w->m;
    M.CGp = CGp;
    M.NG = NG;
    M.k = w->res.k;
    M.row_tiles = (int32_t)((w->n + 127) / 128);
    M.n_tiles = n_tiles;
    items += (int64_t)M.row_tiles * n_tiles;
  }
  // TMA maps of X (box 128 rows x 16 columns); an input TMA cannot read (base not
  // 16-byte aligned or odd leading dimension) is first copied to an aligned buffer
  std::vector<CUtensorMap> maps(nw);
  for (int i = 0; i < nw && ok; ++i) {
    Work* w = ws[i];
    const double* X = static_cast<const double*>(w->X);
    int64_t ldx = w->ldx;
    if (!tma_compatible_f64(X, ldx)) {
      ldx = (w->n + 1) / 2 * 2;
      void* tmp = env.alloc(sizeof(double) * ldx * w->m, "alloc aligned input");
      bufs.push_back(tmp);
      ok = tmp && env.cuda(cudaMemcpy2DAsync(tmp, ldx * sizeof(double), X, w->ldx * sizeof(double),
                                             w->n * sizeof(double), w->m, cudaMemcpyDeviceToDevice, env.s),
                           "copy input for TMA");
      X = static_cast<const double*>(tmp);
      mj[i].X = X;
      mj[i].ldx = ldx;
    }
    if (ok && !encode_colmajor_f64(&maps[i], X, w->n, w->m, ldx, 128, 16))
      ok = env.fail(HAPOD_ERR_CUDA, "cuTensorMapEncodeTiled failed for an X V input");
  }
  double bytes = 0, flops = 0;
  for (Work* w : ws) {
    bytes += 8.0 * w->n * (w->m + w->res.k);
    flops += 2.0 * w->n * w->m * w->res.k;
  }
  cudaEvent_t t0 = env.tic();
  if (ok) {
    OzVSplitJob* vj_d = env.upload(vj, "upload V split jobs");
    OzModesJob* mj_d = env.upload(mj, "upload modes jobs");
    CUtensorMap* maps_d = env.upload(maps, "upload tensor maps");
    bufs.push_back(vj_d);
    bufs.push_back(mj_d);
    bufs.push_back(maps_d);
    ok = vj_d && mj_d && maps_d && env.cuda(launch_oz_vsplit(vj_d, nw, vcols, env.s), "V split launch") &&
         env.cuda(launch_modes_oz(mj_d, maps_d, nw, items, env.err_dev, env.s), "modes launch");
  }
  env.toc(t0, 4, 2, bytes, flops);
  for (void* p : bufs) env.release(p);
  return ok;
}

// ------------------------------------------------------------------ autotuned splits
// Split factor of the Gram planners per (form, m bucket, n bucket), set by
// hapod_autotune; buckets are ceil(log2) of m and n.  100 = the planner's own rule.
std::mutex g_tune_mu;
std::map<std::tuple<int, int, int>, int> g_tune;

int log2_bucket(int64_t v) {
  int b = 0;
  while (b < 62 && ((int64_t)1 << b) < v) ++b;
  return b;
}

// The factor for a batch: that of its widest node (the tiles of the widest node
// dominate the batch's items).
int split_pct_for(int precision, const std::vector<Work*>& ws) {
  const Work* wide = nullptr;
  for (const Work* w : ws)
    if (!wide || w->m > wide->m) wide = w;
  if (!wide) return 100;
  std::lock_guard<std::mutex> lk(g_tune_mu);
  auto it = g_tune.find(std::make_tuple(precision, log2_bucket(wide->m), log2_bucket(wide->n)));
  return it == g_tune.end() ? 100 : it->second;
}

// K1, mixed fixed-point form: 128 x 64 tiles of exact digit products.
bool step_gram_fx3(Env& env, std::vector<Work*>& ws) {
  std::vector<GramJob> jobs(ws.size());
  std::vector<CUtensorMap> maps(2 * ws.size());
  double bytes = 0, flops = 0;
  for (size_t i = 0; i < ws.size(); ++i) {
    // column exponents of this X, for its Gram and the X V that follows (one read of
    // X); always recomputed: a work item may be given another X (CholQR2 passes)
    if (!ws[i]->exps) {
      ws[i]->exps = (int32_t*)env.alloc(sizeof(int32_t) * std::max<int64_t>(1, ws[i]->m), "alloc exponents");
      if (!ws[i]->exps) return false;
    }
    cudaEvent_t tc0 = env.tic();
    const bool okx = env.cuda(launch_fx_colexp(static_cast<const float*>(ws[i]->X), ws[i]->ldx, ws[i]->n, ws[i]->m,
                                               ws[i]->exps, env.s),
                              "column exponent launch");
    env.toc(tc0, 6, 1, 4.0 * ws[i]->n * ws[i]->m, 0.0);
    if (!okx) return false;
    GramJob& J = jobs[i];
    memset(&J, 0, sizeof(J));
    J.col_exp = ws[i]->exps;
    J.X = ws[i]->X;
    J.ldx = ws[i]->ldx;
    J.n = ws[i]->n;
    J.m = (int32_t)ws[i]->m;
    J.G = ws[i]->G;
    if (!encode_colmajor_f32(&maps[2 * i], ws[i]->X, ws[i]->n, ws[i]->m, ws[i]->ldx, gram_fx3_rows_per_stage(),
                             gram_fx3_a_cols(), true) ||
        !encode_colmajor_f32(&maps[2 * i + 1], ws[i]->X, ws[i]->n, ws[i]->m, ws[i]->ldx, gram_fx3_rows_per_stage(),
                             gram_fx3_b_cols(), true))
      return env.fail(HAPOD_ERR_CUDA, "cuTensorMapEncodeTiled failed for a Gram input");
    bytes += 4.0 * ws[i]->n * ws[i]->m;
    flops += (double)ws[i]->n * ws[i]->m * (ws[i]->m + 1);
  }
  std::vector<int4> items, reduce;
  size_t pbytes = 0;
  plan_gram_fx3(jobs.data(), (int)jobs.size(), kNumSMs, items, reduce, &pbytes, split_pct_for(HAPOD_MIXED_FX3, ws));
  GramJob* jobs_d = env.upload(jobs, "upload gram jobs");
  int4* items_d = env.upload(items, "upload gram items");
  int4* red_d = env.upload(reduce, "upload gram reduce");
  CUtensorMap* maps_d = env.upload(maps, "upload tensor maps");
  double* partials = pbytes ? (double*)env.alloc(pbytes, "alloc gram partials") : nullptr;
  bool ok = jobs_d && items_d && red_d && maps_d && (partials || !pbytes) && env.err_dev;
  if (ok) {
    cudaEvent_t t0 = env.tic();
    ok = env.cuda(launch_gram_fx3(jobs_d, maps_d, items_d, (int)items.size(), red_d, (int)reduce.size(), partials,
                                  env.err_dev, env.s),
                  "gram launch");
    env.toc(t0, 0, 1 + !reduce.empty(), bytes, flops);
  }
  env.release(jobs_d);
  env.release(items_d);
  env.release(red_d);
  env.release(maps_d);
  env.release(partials);
  return ok;
}

// K4, mixed fixed-point form: Y = X V_k (diag scale) for every w (k = w->res.k > 0,
// V_k in w->Vk, column exponents in w->exps from the Gram or computed here).
bool step_modes_fx(Env& env, std::vector<Work*>& ws) {
  if (ws.empty()) return true;
  const int nw = (int)ws.size();
  std::vector<FxVSplitJob> vj(nw);
  std::vector<FxModesJob> mj(nw);
  std::vector<CUtensorMap> maps(nw);
  std::vector<void*> bufs;
  int64_t items = 0;
  int max_kpad = 1;
  bool ok = true;
  double bytes = 0, flops = 0;
  for (int i = 0; i < nw && ok; ++i) {
    Work* w = ws[i];
    if (!w->exps) {
      w->exps = (int32_t*)env.alloc(sizeof(int32_t) * std::max<int64_t>(1, w->m), "alloc exponents");
      ok = w->exps && env.cuda(launch_fx_colexp(static_cast<const float*>(w->X), w->ldx, w->n, w->m, w->exps, env.s),
                               "column exponent launch");
      if (!ok) break;
    }
    const int k = w->res.k;
    if (w->m > fx_modes_max_m()) {
      ok = env.fail(HAPOD_ERR_INVALID, "fixed-point X V: more snapshot columns than the form supports");
      break;
    }
    const int mode_tiles = fx_mode_tiles(k), MT = fx_mode_width(k);
    uint16_t* vdig = (uint16_t*)env.alloc(fx_vdig_bytes(w->m, k), "alloc V digits");
    int32_t* fexp = (int32_t*)env.alloc(sizeof(int32_t) * mode_tiles * MT, "alloc mode exponents");
    float2* xscale = (float2*)env.alloc(fx_xscale_bytes(w->m), "alloc column scales");
    float* yscale = (float*)env.alloc(sizeof(float) * mode_tiles * MT * 2, "alloc mode scales");
    float* ymul = yscale ? yscale + mode_tiles * MT : nullptr;
    int32_t* Z = nullptr;
    if (fx_modes_needs_scratch(w->m)) {
      Z = (int32_t*)env.alloc(sizeof(int32_t) * (size_t)w->n * mode_tiles * MT, "alloc X V partial sums");
      bufs.push_back(Z);
      ok = Z != nullptr;
    }
    bufs.push_back(vdig);
    bufs.push_back(fexp);
    bufs.push_back(xscale);
    bufs.push_back(yscale);
    ok = ok && vdig && fexp && xscale && yscale;
    if (!ok) break;
    FxVSplitJob& V = vj[i];
    memset(&V, 0, sizeof(V));
    V.V = w->Vk;
    V.ldv = w->ldvk ? w->ldvk : w->m;
    V.exps = w->exps;
    V.vdig = vdig;
    V.fexp = fexp;
    V.xscale = xscale;
    V.scale = w->scale;
    V.yscale = yscale;
    V.ymul = ymul;
    V.m = (int32_t)w->m;
    V.k = k;
    V.kpad = mode_tiles * MT;
    V.nt = MT;
    max_kpad = std::max(max_kpad, V.kpad);
    FxModesJob& M = mj[i];
    memset(&M, 0, sizeof(M));
    M.X = static_cast<const float*>(w->X);
    M.ldx = w->ldx;
    M.exps = w->exps;
    M.xscale = xscale;
    M.yscale = yscale;
    M.ymul = ymul;
    M.vdig = vdig;
    M.fexp = fexp;
    M.scale = w->scale;
    M.Y = static_cast<float*>(w->Y);
    M.ldy = w->ldy;
    M.n = w->n;
    M.item_base = items;
    M.m = (int32_t)w->m;
    M.k = k;
    M.row_tiles = (int32_t)((w->n + 127) / 128);
    M.mode_tiles = mode_tiles;
    M.nt = MT;
    M.Z = Z;
    M.ldz = w->n;
    items += (int64_t)M.row_tiles * mode_tiles;
    if (!encode_colmajor_f32(&maps[i], w->X, w->n, w->m, w->ldx, 128, 16, false))
      ok = env.fail(HAPOD_ERR_CUDA, "cuTensorMapEncodeTiled failed for an X V input");
    bytes += 4.0 * w->n * (w->m + k);
    flops += 2.0 * w->n * w->m * k;
  }
  cudaEvent_t t0 = env.tic();
  if (ok) {
    FxVSplitJob* vj_d = env.upload(vj, "upload V split jobs");
    FxModesJob* mj_d = env.upload(mj, "upload modes jobs");
    CUtensorMap* maps_d = env.upload(maps, "upload tensor maps");
    bufs.push_back(vj_d);
    bufs.push_back(mj_d);
    bufs.push_back(maps_d);
    ok = vj_d && mj_d && maps_d && env.err_dev &&
         env.cuda(launch_modes_fx(vj_d, nw, max_kpad, mj_d, maps_d, items, env.err_dev, env.s), "modes launch");
  }
  env.toc(t0, 4, 2, bytes, flops);
  for (void* p : bufs) env.release(p);
  return ok;
}

// K1 for every node of ws into w->G.
bool step_gram(Env& env, int precision, std::vector<Work*>& ws) {
  if (ws.empty()) return true;
  if (precision == HAPOD_FP64_OZAKI) return step_gram_oz(env, ws);
  if (precision == HAPOD_MIXED_FX3) return step_gram_fx3(env, ws);
  const bool fp64 = precision == HAPOD_FP64;
  const bool bf3 = precision == HAPOD_MIXED_BF16X3;
  std::vector<GramJob> jobs(ws.size());
  for (size_t i = 0; i < ws.size(); ++i) {
    GramJob& J = jobs[i];
    memset(&J, 0, sizeof(J));
    J.X = ws[i]->X;
    J.ldx = ws[i]->ldx;
    J.n = ws[i]->n;
    J.m = (int32_t)ws[i]->m;
    J.G = ws[i]->G;
  }
  int4 *items = nullptr, *reduce = nullptr;
  GramPlan plan;
  const int tile = fp64 ? 64 : 128;
  // concurrent CTAs: four 256-thread FP64 CTAs per SM, one tensor-core CTA per SM;
  // items of at least 256 (FP64) / 2048 (tensor-core) rows
  plan_gram(jobs.data(), (int)jobs.size(), tile, fp64 ? 256 : 2048, fp64 ? 4 * kNumSMs : kNumSMs, &items, &reduce,
            &plan, !fp64, split_pct_for(precision, ws));
  std::vector<int4> it(items, items + plan.num_items), rd(reduce, reduce + plan.num_reduce);
  free(items);
  std::vector<CUtensorMap> maps;
  if (!fp64) {
    maps.resize(ws.size());
    for (size_t i = 0; i < ws.size(); ++i)
      if (!encode_colmajor_f32(&maps[i], ws[i]->X, ws[i]->n, ws[i]->m, ws[i]->ldx,
                               bf3 ? gram_bf3_rows_per_stage() : gram_tc_rows_per_stage(), 128, true))
        return env.fail(HAPOD_ERR_CUDA, "cuTensorMapEncodeTiled failed for a Gram input");
  }
  GramJob* jobs_d = env.upload(jobs, "upload gram jobs");
  int4* items_d = env.upload(it, "upload gram items");
  int4* red_d = env.upload(rd, "upload gram reduce");
  CUtensorMap* maps_d = fp64 ? nullptr : env.upload(maps, "upload tensor maps");
  double* partials = plan.partial_bytes ? (double*)env.alloc(plan.partial_bytes, "alloc gram partials") : nullptr;
  int* errf = fp64 ? nullptr : env.err_dev;
  bool ok = jobs_d && items_d && red_d && (partials || !plan.partial_bytes) && (fp64 || (errf && maps_d));
  if (ok) {
    cudaError_t e;
    double bytes = 0, flops = 0;
    for (Work* w : ws) {
      bytes += (double)elem_size(precision) * w->n * w->m;
      flops += (double)w->n * w->m * (w->m + 1);
    }
    cudaEvent_t t0 = env.tic();
    if (fp64)
      e = launch_gram_f64(jobs_d, items_d, plan.num_items, red_d, plan.num_reduce, partials, env.s);
    else if (bf3)
      e = launch_gram_bf3(jobs_d, maps_d, items_d, plan.num_items, red_d, plan.num_reduce, partials, errf, env.s);
    else
      e = launch_gram_tc(jobs_d, maps_d, items_d, plan.num_items, red_d, plan.num_reduce, partials, errf, env.s);
    env.toc(t0, 0, 1 + (plan.num_reduce > 0), bytes, flops);
    ok = ok && env.cuda(e, "gram launch");
  }
  env.release(jobs_d);
  env.release(items_d);
  env.release(red_d);
  env.release(maps_d);
  env.release(partials);
  return ok;
}

// Eigensolver variant of a form: FP32 rotations for the mixed TF32 form, FP64 rotations
// for every other form.
// FP64-data forms rotate in FP64; the mixed forms with FP64 eigenvectors in double-float
int eig_mode(int precision) {
  return precision == HAPOD_MIXED_TF32X3 ? kEigF32 : f64_data(precision) ? kEigF64 : kEigDF;
}
// Relative level of a form's Gram error (the pivoted Cholesky does not factor below it).
double gram_floor_rel(int precision) {
  return precision == HAPOD_MIXED_BF16X3 ? 1e-10 : precision == HAPOD_MIXED_FX3 ? 1e-13 : 0.0;
}
// Eigenvectors are stored in FP64 except by the mixed TF32 form (FP32).
bool eigvec_f64(int precision) { return precision != HAPOD_MIXED_TF32X3; }

// K2 for every node (w->G -> lambda, perm, V); results land in res_d[i].
bool step_eig(Env& env, int precision, std::vector<Work*>& ws, NodeResult* res_d) {
  if (ws.empty()) return true;
  std::vector<EigJob> jobs(ws.size());
  int max_m = 1;
  for (size_t i = 0; i < ws.size(); ++i) {
    Work* w = ws[i];
    if (w->m > kEigMaxM) return env.fail(HAPOD_ERR_INVALID, "node wider than the eigensolver supports (13000 columns)");
    EigJob& J = jobs[i];
    memset(&J, 0, sizeof(J));
    J.G = w->G;
    J.A = w->A;
    J.V = w->V;
    J.lam_tmp = w->lam_tmp;
    J.lambda = w->lambda;
    J.perm = w->perm;
    J.result = res_d + i;
    J.eps2 = w->eps * w->eps;
    J.floor_rel = gram_floor_rel(precision);
    J.m = (int32_t)w->m;
    max_m = std::max(max_m, (int)w->m);
  }
  EigJob* jobs_d = (EigJob*)env.alloc(sizeof(EigJob) * jobs.size(), "alloc eig jobs");
  EigSync* sync_d = (EigSync*)env.alloc(sizeof(EigSync) * jobs.size(), "alloc eig barriers");
  bool ok = jobs_d && sync_d;
  cudaEvent_t t0 = env.tic();
  ok = ok && env.cuda(launch_eig(eig_mode(precision), jobs.data(), jobs_d, (int)jobs.size(), max_m, kMaxSweeps,
                                 sync_d, env.err_dev, env.s, env.stage),
                      "eigensolver launch");
  env.toc(t0, 1, 1, 0.0, 0.0);
  env.release(jobs_d);
  env.release(sync_d);
  return ok;
}

bool step_truncate(Env& env, std::vector<Work*>& ws, NodeResult* res_d) {
  if (ws.empty()) return true;
  std::vector<TruncJob> jobs(ws.size());
  for (size_t i = 0; i < ws.size(); ++i) {
    jobs[i].lambda = ws[i]->lambda;
    jobs[i].sigma = ws[i]->sigma;
    jobs[i].result = res_d + i;
    jobs[i].eps2 = ws[i]->eps * ws[i]->eps;
    jobs[i].m = (int32_t)ws[i]->m;
    jobs[i].pad = 0;
  }
  TruncJob* d = env.upload(jobs, "upload trunc jobs");
  cudaEvent_t t0 = env.tic();
  bool ok = d && env.cuda(launch_truncate(d, (int)jobs.size(), env.s), "truncate launch");
  env.toc(t0, 2, 1, 0.0, 0.0);
  env.release(d);
  return ok;
}

// Gram + eig + truncation for ws, then read back k, tail, sigma (synchronises).
bool run_pod_front(Env& env, int precision, std::vector<Work*>& ws) {
  if (ws.empty()) return true;
  const bool fp64 = f64_data(precision);
  if (!alloc_work(env, ws, eigvec_f64(precision))) return false;
  if (!fp64) {
    // TMA reads need a 16-byte aligned base and pitch; copy the rare input that has neither
    for (Work* w : ws) {
      if (tma_compatible_f32(w->X, w->ldx)) continue;
      const int64_t ld = (w->n + 31) / 32 * 32;
      w->X_tmp = env.alloc(sizeof(float) * ld * w->m, "alloc aligned input");
      if (!w->X_tmp) return false;
      if (!env.cuda(cudaMemcpy2DAsync(w->X_tmp, ld * sizeof(float), w->X, w->ldx * sizeof(float),
                                      w->n * sizeof(float), w->m, cudaMemcpyDeviceToDevice, env.s),
                    "copy input for TMA"))
        return false;
      w->X = w->X_tmp;
      w->ldx = ld;
    }
  }
  NodeResult* res_d = (NodeResult*)env.alloc(sizeof(NodeResult) * ws.size() + sizeof(int) * 4, "alloc results");
  if (!res_d) return false;
  env.err_dev = reinterpret_cast<int*>(res_d + ws.size());
  bool ok = env.cuda(cudaMemsetAsync(res_d, 0, sizeof(NodeResult) * ws.size() + sizeof(int) * 4, env.s), "memset") &&
            init_err_flag(env, env.err_dev);
  ok = ok && step_gram(env, precision, ws);
  ok = ok && step_eig(env, precision, ws, res_d);
  ok = ok && step_truncate(env, ws, res_d);
  std::vector<NodeResult> res(ws.size());
  int dev_err = 0;
  if (ok)
    ok = env.cuda(cudaMemcpyAsync(res.data(), res_d, sizeof(NodeResult) * ws.size(), cudaMemcpyDeviceToHost, env.s),
                  "read back results") &&
         env.cuda(cudaMemcpyAsync(&dev_err, env.err_dev, sizeof(int), cudaMemcpyDeviceToHost, env.s), "read back flag");
  for (Work* w : ws) {
    w->sigma_host.assign((size_t)w->m, 0.0);
    if (ok)
      ok = env.cuda(cudaMemcpyAsync(w->sigma_host.data(), w->sigma, sizeof(double) * w->m, cudaMemcpyDeviceToHost,
                                    env.s),
                    "read back sigma");
  }
  ok = ok && env.cuda(cudaStreamSynchronize(env.s), "synchronize");
  env.release(res_d);
  env.err_dev = nullptr;
  if (!ok) return false;
  if (dev_err) return env.fail(HAPOD_ERR_TIMEOUT, "device-side wait timed out in the tensor-core Gram kernel");
  for (size_t i = 0; i < ws.size(); ++i) {
    ws[i]->res = res[i];
    ws[i]->sigma_host.resize((size_t)std::max(0, res[i].k));
    const int st = res[i].status;
    if (st != HAPOD_OK && st < HAPOD_WARN_NOCONVERGE)
      return env.fail((hapod_status)st, st == HAPOD_ERR_NONFINITE ? "non-finite value in a Gram matrix"
                                                                   : "device-side wait timed out in the eigensolver");
  }
  return true;
}

// Gather V_k and form Y = X V_k (diag(scale)) into w->Y for every w with k > 0.
bool run_pod_back(Env& env, int precision, std::vector<Work*>& ws) {
  const bool fp64 = f64_data(precision);
  std::vector<GatherJob> gj;
  std::vector<ModesJob> mj;
  std::vector<Work*> act;
  for (Work* w : ws)
    if (w->res.k > 0 && w->Y) act.push_back(w);
  if (act.empty()) return true;
  for (Work* w : act) {
    w->Vk = (double*)env.alloc(sizeof(double) * w->m * w->res.k, "alloc Vk");
    if (!w->Vk) return false;
    GatherJob g;
    g.V = w->V;
    g.perm = w->perm;
    g.Vk = w->Vk;
    g.m = (int32_t)w->m;
    g.k = w->res.k;
    gj.push_back(g);
  }
  GatherJob* gd = env.upload(gj, "upload gather jobs");
  cudaEvent_t tg = env.tic();
  bool ok = gd && env.cuda(launch_gather(eigvec_f64(precision), gd, (int)gj.size(), env.s), "gather launch");
  env.toc(tg, 3, 1, 0.0, 0.0);
  env.release(gd);
  if (!ok) return false;
  if (precision == HAPOD_FP64_OZAKI || precision == HAPOD_MIXED_FX3) {
    // tensor-core X V with bounded waits: an error flag of its own, read back here
    int* prev = env.err_dev;
    int* flag = prev;
    if (!flag) {
      flag = (int*)env.alloc(sizeof(int) * 2, "alloc flag");
      if (!flag || !env.cuda(cudaMemsetAsync(flag, 0, sizeof(int) * 2, env.s), "memset") ||
          !init_err_flag(env, flag)) {
        env.release(prev ? nullptr : flag);
        return false;
      }
      env.err_dev = flag;
    }
    ok = precision == HAPOD_FP64_OZAKI ? step_modes_oz(env, act) : step_modes_fx(env, act);
    int dev_err = 0;
    if (ok && !prev)
      ok = env.cuda(cudaMemcpyAsync(&dev_err, flag, sizeof(int), cudaMemcpyDeviceToHost, env.s), "read flag") &&
           env.cuda(cudaStreamSynchronize(env.s), "synchronize");
    if (!prev) {
      env.release(flag);
      env.err_dev = nullptr;
    }
    if (ok && dev_err) return env.fail(HAPOD_ERR_TIMEOUT, "device-side wait timed out in the tensor-core X V kernel");
    return ok;
  }
  int max_k = 0;
  for (Work* w : act) max_k = std::max(max_k, w->res.k);
  const int tr = fp64 ? modes_f64_tile_rows(max_k) : modes_mixed_rows_per_block(max_k);
  const int tc = fp64 ? modes_f64_tile_cols(max_k) : modes_mixed_tile_cols(max_k);
  int64_t blocks = 0;
  for (Work* w : act) {
    ModesJob J;
    memset(&J, 0, sizeof(J));
    J.X = w->X;
    J.ldx = w->ldx;
    J.Vk = w->Vk;
    J.ldv = w->m;
    J.scale = w->scale;
    J.Y = w->Y;
    J.ldy = w->ldy;
    J.n = w->n;
    J.m = (int32_t)w->m;
    J.k = w->res.k;
    J.row_tiles = (int32_t)((w->n + tr - 1) / tr);
    J.col_tiles = (J.k + tc - 1) / tc;
    J.block_base = blocks;
    blocks += (int64_t)J.row_tiles * J.col_tiles;
    mj.push_back(J);
  }
  ModesJob* md = env.upload(mj, "upload modes jobs");
  if (!md) return false;
  double bytes = 0, flops = 0;
  const size_t es = fp64 ? sizeof(double) : sizeof(float);
  for (Work* w : act) {
    bytes += (double)es * w->n * (w->m + w->res.k);
    flops += 2.0 * w->n * w->m * w->res.k;
  }
  if (fp64) {
    cudaEvent_t t0 = env.tic();
    ok = env.cuda(launch_modes_f64(md, (int)mj.size(), blocks, tc, env.s), "modes launch");
    env.toc(t0, 4, 1, bytes, flops);
  } else {
    bool vec = true;
    for (const ModesJob& J : mj) vec = vec && tma_compatible_f32(J.X, J.ldx) && tma_compatible_f32(J.Y, J.ldy);
    cudaEvent_t t0 = env.tic();
    ok = env.cuda(launch_modes_mixed(md, (int)mj.size(), blocks, tc, vec, env.s), "modes launch");
    env.toc(t0, 4, 1, bytes, flops);
  }
  env.release(md);
  return ok;
}

// Y (n x m, FP32, ld ldx) -> Out = Y M (n x k), M FP64 m x k (ld m): one mixed modes launch.
bool modes_pass_mixed(Env& env, const void* X, int64_t ldx, int64_t n, int m, const double* M, int k, void* Out,
                      int64_t ldo) {
  ModesJob J;
  memset(&J, 0, sizeof(J));
  J.X = X;
  J.ldx = ldx;
  J.Vk = M;
  J.ldv = m;
  J.Y = Out;
  J.ldy = ldo;
  J.n = n;
  J.m = m;
  J.k = k;
  J.row_tiles = (int32_t)((n + modes_mixed_rows_per_block(k) - 1) / modes_mixed_rows_per_block(k));
  J.col_tiles = (k + modes_mixed_tile_cols(k) - 1) / modes_mixed_tile_cols(k);
  std::vector<ModesJob> mj{J};
  ModesJob* md = env.upload(mj, "upload modes job");
  if (!md) return false;
  const bool vec = tma_compatible_f32(X, ldx) && tma_compatible_f32(Out, ldo);
  cudaEvent_t t0 = env.tic();
  bool ok = env.cuda(launch_modes_mixed(md, 1, (int64_t)J.row_tiles * J.col_tiles, modes_mixed_tile_cols(k), vec,
                                        env.s),
                     "modes launch");
  env.toc(t0, 4, 1, 4.0 * n * (m + k), 2.0 * n * m * k);
  env.release(md);
  return ok;
}

// CholQR2 of the root's sigma-scaled modes Y (mixed form): U (orthonormal columns,
// written to `out`) and refreshed sigma (host).  Sec. 2 footnote of the
// method-of-snapshots remark: the Gram route loses orthogonality as cond(X)^2.
bool root_cholqr2(Env& env, int precision, const void* Y, int64_t n, int64_t ldn, int k, void* out,
                  std::vector<double>& sigma, bool* rank_deficient) {
  const size_t kk = (size_t)k * k;
  // layout (doubles): W | W2 | R1 | M1 | M | work (4 k^2) | sigma (k)
  double* W = (double*)env.alloc(sizeof(double) * (9 * kk + k), "alloc CholQR2 work");
  void* Q1 = env.alloc(sizeof(float) * ldn * k, "alloc CholQR2 Q1");
  int* flag = (int*)env.alloc(sizeof(int) * 4, "alloc flag");
  if (!W || !Q1 || !flag) return false;
  double *W2 = W + kk, *R1 = W + 2 * kk, *M1 = W + 3 * kk, *M = W + 4 * kk, *work = W + 5 * kk;
  double* sig_d = W + 9 * kk;
  bool ok = env.cuda(cudaMemsetAsync(flag, 0, sizeof(int) * 4, env.s), "memset") && init_err_flag(env, flag + 1);
  Work g;
  g.X = Y;
  g.ldx = ldn;
  g.n = n;
  g.m = k;
  g.G = W;
  std::vector<Work*> ws{&g};
  env.err_dev = flag + 1;
  ok = ok && step_gram(env, precision, ws);
  ok = ok && env.cuda(launch_cholqr_first(W, R1, M1, k, flag, env.s), "cholqr launch");
  ok = ok && modes_pass_mixed(env, Y, ldn, n, k, M1, k, Q1, ldn);
  g.X = Q1;
  g.G = W2;
  ok = ok && step_gram(env, precision, ws);
  ok = ok && env.cuda(launch_cholqr_second(W2, R1, work, M, sig_d, k, flag, env.s), "cholqr launch");
  ok = ok && modes_pass_mixed(env, Q1, ldn, n, k, M, k, out, ldn);
  int hflag[2] = {0, 0};
  sigma.assign((size_t)k, 0.0);
  if (ok)
    ok = env.cuda(cudaMemcpyAsync(sigma.data(), sig_d, sizeof(double) * k, cudaMemcpyDeviceToHost, env.s), "read") &&
         env.cuda(cudaMemcpyAsync(hflag, flag, sizeof(int) * 2, cudaMemcpyDeviceToHost, env.s), "read") &&
         env.cuda(cudaStreamSynchronize(env.s), "synchronize");
  env.err_dev = nullptr;
  env.release(W);
  env.release(Q1);
  env.release(flag);
  if (!ok) return false;
  if (hflag[1]) return env.fail(HAPOD_ERR_TIMEOUT, "device-side wait timed out in the tensor-core Gram kernel");
  *rank_deficient = hflag[0] != 0;
  return true;
}

}  // namespace

void hapod::set_thread_error(const char* msg) { g_thread_error = msg; }

// ====================================================================== context
struct NodeRT {
  int32_t parent = -1;
  std::vector<int32_t> children;
  int32_t level = 1;
  int64_t leaf_cols = 0;
  int64_t acc = 0;
  double eps = 0.0;
  int state = 0;  // 0 waiting, 1 ready, 2 done
  // input
  const void* in = nullptr;
  int64_t in_ld = 0;
  int64_t m = 0;
  void* in_owned = nullptr;
  // as a parent: input buffer being filled by the children
  void* pbuf = nullptr;
  int64_t pfill = 0;
  int children_done = 0;
  // output
  int64_t k = -1;
  double tail = 0.0;
  int32_t sweeps = 0;
  int32_t status = HAPOD_OK;
  std::vector<double> sigma;
  void* stash = nullptr;  // own copy of the output while the parent cannot be sized
  int64_t stash_offset = -1;
  // right singular vectors (HAPOD_FLAG_RIGHT_VECTORS): V_N (m x k FP64, null at
  // pass-through nodes: the identity) and the first column of this node's modes in
  // its parent's input
  double* rv = nullptr;
  int64_t pcol = -1;
};

constexpr size_t kStageBytes = (size_t)8 << 20;  // pinned staging arena of a context

struct hapod_ctx {
  Env env;
  HostStage stage;
  Prof* prof = nullptr;
  int64_t n = 0;
  int64_t ldn = 0;  // leading dimension of library-owned node buffers (n rounded up to 32)
  int precision = HAPOD_FP64;
  size_t esize = 8;
  std::vector<NodeRT> nodes;
  int root = -1;
  int LT = 1;
  int64_t S = 0;
  double eps_star = 0.0;
  int max_pending = 0;
  bool keep_rv = false;
  int pending = 0;
  int leaves_total = 0;
  int leaves_pushed = 0;
  bool poisoned = false;
  hapod_status warning = HAPOD_OK;
  void* result = nullptr;  // n x k root modes (phi), owned
  std::string err = "no error";
};

namespace {

hapod_status ctx_fail(hapod_ctx* c) {
  c->poisoned = true;
  c->err = c->env.err;
  return c->env.code;
}

// Allocate parent p's input buffer once every child's rank is known (sized
// exactly: sum of the children's k) and move in the outputs that children of
// earlier batches parked in their own buffers.  Returns false on failure.
bool ensure_parent_buffer(hapod_ctx* c, int p) {
  NodeRT& P = c->nodes[p];
  if (P.pbuf) return true;
  const size_t col_bytes = (size_t)c->ldn * c->esize;
  int64_t cap = 0;
  for (int ch : P.children) cap += std::max<int64_t>(0, c->nodes[ch].k);
  if (cap == 0) return true;
  P.pbuf = c->env.alloc(col_bytes * cap, "alloc parent input");
  if (!P.pbuf) return false;
  for (int ch : P.children) {
    NodeRT& C = c->nodes[ch];
    if (C.state == 2 && C.stash && C.k > 0) {
      if (!c->env.cuda(cudaMemcpyAsync((char*)P.pbuf + (size_t)P.pfill * col_bytes, C.stash, C.k * col_bytes,
                                       cudaMemcpyDeviceToDevice, c->env.s),
                       "copy parked modes"))
        return false;
      C.pcol = P.pfill;
      P.pfill += C.k;
      c->env.release(C.stash);
      C.stash = nullptr;
    }
  }
  return true;
}

// Where the output of node a (k > 0) goes once its rank is known: the root's
// result buffer, its slot in the parent's input buffer when every sibling's rank
// is known in this batch, or else a parked buffer of its own.  Returns the device
// pointer of its first column (ld = n), or nullptr on allocation failure.
void* place_output(hapod_ctx* c, int a, const std::vector<int>& batch_children) {
  NodeRT& A = c->nodes[a];
  const size_t col_bytes = (size_t)c->ldn * c->esize;
  if (A.parent < 0) {
    c->result = c->env.alloc(col_bytes * std::max<int64_t>(1, A.k), "alloc result");
    return c->result;
  }
  NodeRT& P = c->nodes[A.parent];
  if (P.children_done + batch_children[A.parent] == (int)P.children.size()) {
    if (!ensure_parent_buffer(c, A.parent)) return nullptr;
    void* dst = (char*)P.pbuf + (size_t)P.pfill * col_bytes;
    A.pcol = P.pfill;
    P.pfill += A.k;
    return dst;
  }
  A.stash = c->env.alloc(col_bytes * A.k, "alloc parked modes");
  return A.stash;
}

bool run_batch(hapod_ctx* c, const std::vector<int>& batch) {
  Env& env = c->env;
  const size_t col_bytes = (size_t)c->n * c->esize;    // bytes of one column
  const size_t pitch = (size_t)c->ldn * c->esize;      // column pitch of library buffers
  std::vector<Work> works(batch.size());
  std::vector<Work*> compute;
  for (size_t i = 0; i < batch.size(); ++i) {
    NodeRT& A = c->nodes[batch[i]];
    Work& w = works[i];
    w.X = A.in;
    w.ldx = A.in_ld;
    w.n = c->n;
    w.m = A.m;
    w.eps = A.eps;
    if (A.eps > 0.0 && A.m > 0) compute.push_back(&w);
  }
  if (!run_pod_front(env, c->precision, compute)) {
    free_work(env, compute);
    return false;
  }
  // ranks known: pass-through (eps = 0) keeps all m columns with sigma = 1 (Def. truncated POD)
  std::vector<int> batch_children(c->nodes.size(), 0);
  for (size_t i = 0; i < batch.size(); ++i) {
    NodeRT& A = c->nodes[batch[i]];
    Work& w = works[i];
    if (A.eps > 0.0 && A.m > 0) {
      A.k = w.res.k;
      A.tail = w.res.tail;
      A.sweeps = w.res.sweeps;
      A.status = w.res.status;
      A.sigma = w.sigma_host;
      if (A.status >= HAPOD_WARN_NOCONVERGE && c->warning == HAPOD_OK) c->warning = (hapod_status)A.status;
    } else {
      A.k = A.m;
      A.tail = 0.0;
      A.sweeps = 0;
      A.sigma.assign((size_t)A.m, 1.0);
    }
    if (A.parent >= 0) batch_children[A.parent]++;
  }
  // output placement and modes
  bool ok = true;
  std::vector<double*> scales;
  void* root_tmp = nullptr;
  Work* root_work = nullptr;
  int root_node = -1;
  for (size_t i = 0; i < batch.size() && ok; ++i) {
    const int a = batch[i];
    NodeRT& A = c->nodes[a];
    Work& w = works[i];
    if (A.k <= 0) {
      if (A.parent < 0) c->result = nullptr;
      continue;
    }
    void* dst = place_output(c, a, batch_children);
    if (!dst) {
      ok = false;
      break;
    }
    if (A.eps > 0.0 && A.m > 0) {
      w.Y = dst;
      w.ldy = c->ldn;
      if (A.parent < 0 && mixed_form(c->precision) && A.k <= 256) {
        // mixed form: unscaled Y to a temporary; CholQR2 writes U into the result below
        root_tmp = env.alloc(pitch * A.k, "alloc root modes");
        if (!root_tmp) {
          ok = false;
          break;
        }
        w.Y = root_tmp;
        root_work = &w;
        root_node = batch[i];
      } else if (A.parent < 0) {
        std::vector<double> inv(A.k);
        for (int64_t j = 0; j < A.k; ++j) inv[j] = 1.0 / A.sigma[j];
        w.scale = env.upload(inv, "upload scale");
        if (!w.scale) ok = false;
        scales.push_back(w.scale);
        // resolution floor of the method of snapshots (Sec. 2 footnote: cond(G) = cond(X)^2)
        const double u = f64_data(c->precision)                    ? 1.1102230246251565e-16
                         : gram_floor_rel(c->precision) > 0.0 ? gram_floor_rel(c->precision)
                                                              : 5.9604644775390625e-08;
        if (A.sigma[A.k - 1] < A.sigma[0] * std::sqrt((double)A.m * u)) {
          A.status = HAPOD_WARN_BELOW_FLOOR;
          if (c->warning == HAPOD_OK) c->warning = HAPOD_WARN_BELOW_FLOOR;
        }
      }
    } else {
      cudaEvent_t t0 = env.tic();
      ok = env.cuda(cudaMemcpy2DAsync(dst, pitch, A.in, (size_t)A.in_ld * c->esize, col_bytes, (size_t)A.m,
                                      cudaMemcpyDeviceToDevice, env.s),
                    "copy pass-through snapshots");
      env.toc(t0, 5, 0, 2.0 * col_bytes * A.m, 0.0);
    }
  }
  if (ok) ok = run_pod_back(env, c->precision, compute);
  if (ok && c->keep_rv) {  // keep V_N of every computed node for hapod_result_right
    for (size_t i = 0; i < batch.size() && ok; ++i) {
      NodeRT& A = c->nodes[batch[i]];
      Work& w = works[i];
      if (!(A.eps > 0.0 && A.m > 0 && A.k > 0) || !w.Vk) continue;
      A.rv = (double*)env.alloc(sizeof(double) * (size_t)A.m * (size_t)A.k, "alloc right vectors");
      ok = A.rv && env.cuda(cudaMemcpyAsync(A.rv, w.Vk, sizeof(double) * (size_t)A.m * (size_t)A.k,
                                            cudaMemcpyDeviceToDevice, env.s),
                            "keep right vectors");
    }
  }
  if (ok && root_work) {
    NodeRT& R = c->nodes[root_node];
    bool deficient = false;
    // the fixed-point form keeps the eigensolver's singular values (FP64 eigenvalues of a
    // Gram matrix exact to the representation of the data); CholQR2 orthonormalises U
    std::vector<double> sig_keep = R.sigma;
    ok = root_cholqr2(env, c->precision, root_tmp, c->n, c->ldn, (int)R.k, c->result, R.sigma, &deficient);
    if (c->precision == HAPOD_MIXED_FX3) R.sigma = sig_keep;
    if (ok && deficient) {
      R.status = HAPOD_WARN_BELOW_FLOOR;
      if (c->warning == HAPOD_OK) c->warning = HAPOD_WARN_BELOW_FLOOR;
    }
  }
  env.release(root_tmp);
  free_work(env, compute);
  for (double* s : scales) env.release(s);
  if (!ok) return false;
  // bookkeeping: free owned inputs, mark done, promote parents
  for (size_t i = 0; i < batch.size(); ++i) {
    NodeRT& A = c->nodes[batch[i]];
    if (A.in_owned) {
      env.release(A.in_owned);
      A.in_owned = nullptr;
    }
    A.in = nullptr;
    A.state = 2;
  }
  for (size_t i = 0; i < batch.size(); ++i) {
    NodeRT& A = c->nodes[batch[i]];
    if (A.parent < 0) continue;
    NodeRT& P = c->nodes[A.parent];
    P.children_done++;
    if (P.children_done == (int)P.children.size()) {
      if (!ensure_parent_buffer(c, A.parent)) return false;  // last children may all have kept 0 modes
      P.state = 1;
      P.in = P.pbuf;
      P.in_owned = P.pbuf;
      P.in_ld = c->ldn;
      P.m = P.pfill;
      P.pbuf = nullptr;
    }
  }
  return true;
}

hapod_status run_ready(hapod_ctx* c) {
  for (;;) {
    std::vector<int> batch;
    for (int a = 0; a < (int)c->nodes.size(); ++a)
      if (c->nodes[a].state == 1) batch.push_back(a);
    if (batch.empty()) break;
    for (int a : batch)
      if (c->nodes[a].children.empty()) c->pending--;
    if (!run_batch(c, batch)) return ctx_fail(c);
  }
  return HAPOD_OK;
}

}  // namespace

// ====================================================================== ABI
extern "C" {

hapod_status hapod_create(const hapod_tree* tree, const hapod_tol* tol, int64_t n_rows, void* stream,
                          hapod_ctx** out) {
  if (out) *out = nullptr;
  if (!tree || !tol || !out || !tree->parent || !tree->leaf_cols || tree->num_nodes < 1 || n_rows < 1) {
    g_thread_error = "hapod_create: null argument or non-positive size";
    return HAPOD_ERR_INVALID;
  }
  if (!(tol->eps >= 0.0) || !(tol->omega >= 0.0 && tol->omega <= 1.0) || !valid_precision(tol->precision) ||
      tol->max_pending_leaves < 0) {
    g_thread_error = "hapod_create: eps < 0, omega outside [0, 1], unknown precision or negative max_pending_leaves";
    return HAPOD_ERR_INVALID;
  }
  const int N = tree->num_nodes;
  hapod_ctx* c = new (std::nothrow) hapod_ctx();
  if (!c) {
    g_thread_error = "hapod_create: out of host memory";
    return HAPOD_ERR_OOM;
  }
  c->nodes.resize(N);
  // Def. Rooted Tree: one root, each node a child of at most one node (parent array), all reach the root
  for (int a = 0; a < N; ++a) {
    const int p = tree->parent[a];
    if (p < -1 || p >= N || p == a) {
      g_thread_error = "hapod_create: parent index out of range";
      delete c;
      return HAPOD_ERR_TREE;
    }
    c->nodes[a].parent = p;
    if (p < 0) {
      if (c->root >= 0) {
        g_thread_error = "hapod_create: more than one root";
        delete c;
        return HAPOD_ERR_TREE;
      }
      c->root = a;
    } else {
      c->nodes[p].children.push_back(a);
    }
  }
  if (c->root < 0) {
    g_thread_error = "hapod_create: no root (parent == -1)";
    delete c;
    return HAPOD_ERR_TREE;
  }
  // connectivity (Eq. treeconnected): post-order from the root must reach all nodes
  std::vector<int> order;
  order.reserve(N);
  {
    std::vector<std::pair<int, bool>> st{{c->root, false}};
    std::vector<char> seen(N, 0);
    while (!st.empty()) {
      auto [a, done] = st.back();
      st.pop_back();
      if (done) {
        order.push_back(a);
        continue;
      }
      if (seen[a]) continue;
      seen[a] = 1;
      st.push_back({a, true});
      for (int ch : c->nodes[a].children) st.push_back({ch, false});
    }
    if ((int)order.size() != N) {
      g_thread_error = "hapod_create: some nodes do not reach the root (cycle or disconnected)";
      delete c;
      return HAPOD_ERR_TREE;
    }
  }
  // levels L_T(a) and |S~_a| (post-order)
  for (int a : order) {
    NodeRT& A = c->nodes[a];
    if (A.children.empty()) {
      A.level = 1;
      if (tree->leaf_cols[a] < 0) {
        g_thread_error = "hapod_create: negative leaf_cols";
        delete c;
        return HAPOD_ERR_INVALID;
      }
      A.leaf_cols = tree->leaf_cols[a];
      A.acc = A.leaf_cols;
      c->leaves_total++;
    } else {
      int lv = 0;
      int64_t acc = 0;
      for (int ch : A.children) {
        lv = std::max(lv, c->nodes[ch].level);
        acc += c->nodes[ch].acc;
      }
      A.level = lv + 1;
      A.acc = acc;
    }
  }
  c->LT = c->nodes[c->root].level;
  c->S = c->nodes[c->root].acc;
  c->eps_star = c->S > 0 ? tol->eps / std::sqrt((double)c->S) : 0.0;
  // Thm. cor:hapod_bound; a single-node tree gives its root the whole budget
  for (int a = 0; a < N; ++a) {
    NodeRT& A = c->nodes[a];
    if (a == c->root)
      A.eps = std::sqrt((double)A.acc) * (c->LT > 1 ? tol->omega : 1.0) * c->eps_star;
    else
      A.eps = std::sqrt((double)A.acc) / std::sqrt((double)(c->LT - 1)) *
              std::sqrt(std::max(0.0, 1.0 - tol->omega * tol->omega)) * c->eps_star;
    if (tol->eps_override && !std::isnan(tol->eps_override[a])) {
      if (!(tol->eps_override[a] >= 0.0)) {
        g_thread_error = "hapod_create: negative eps_override";
        delete c;
        return HAPOD_ERR_INVALID;
      }
      A.eps = tol->eps_override[a];
    }
  }
  c->n = n_rows;
  c->ldn = (n_rows + 31) / 32 * 32;
  c->precision = tol->precision;
  c->esize = elem_size(tol->precision);
  c->max_pending = tol->max_pending_leaves;
  c->keep_rv = (tol->flags & HAPOD_FLAG_RIGHT_VECTORS) != 0;
  if (tol->flags & HAPOD_FLAG_PROFILE) {
    c->prof = new (std::nothrow) Prof();
    c->env.prof = c->prof;
  }
  if (!init_env(c->env, stream)) {
    g_thread_error = c->env.err;
    hapod_status st = c->env.code;
    delete c->prof;
    delete c;
    return st;
  }
  // staging arena for the job tables (without it uploads use cudaMemcpyAsync)
  void* stage = nullptr;
  if (cudaHostAlloc(&stage, kStageBytes, cudaHostAllocMapped | cudaHostAllocPortable) == cudaSuccess) {
    c->stage.base = static_cast<uint8_t*>(stage);
    c->stage.cap = kStageBytes;
    c->env.stage = &c->stage;
  } else {
    cudaGetLastError();
  }
  *out = c;
  return HAPOD_OK;
}

hapod_status hapod_push(hapod_ctx* c, int32_t leaf, const void* dev_snapshots, int64_t ld, int64_t ncols) {
  if (!c) {
    g_thread_error = "hapod_push: null context";
    return HAPOD_ERR_INVALID;
  }
  if (c->poisoned) return HAPOD_ERR_STATE;
  if (leaf < 0 || leaf >= (int)c->nodes.size()) {
    c->err = "hapod_push: node index out of range";
    return HAPOD_ERR_INVALID;
  }
  NodeRT& A = c->nodes[leaf];
  if (!A.children.empty()) {
    c->err = "hapod_push: node is not a leaf";
    return HAPOD_ERR_STATE;
  }
  if (A.state != 0) {
    c->err = "hapod_push: leaf already pushed";
    return HAPOD_ERR_STATE;
  }
  if (ncols != A.leaf_cols || (ncols > 0 && (!dev_snapshots || ld < c->n))) {
    c->err = "hapod_push: ncols differs from leaf_cols, null pointer or ld < n";
    return HAPOD_ERR_INVALID;
  }
  A.in = dev_snapshots;
  A.in_ld = ld;
  A.m = ncols;
  A.state = 1;
  c->leaves_pushed++;
  c->pending++;
  const bool all = c->leaves_pushed == c->leaves_total;
  if (all || (c->max_pending > 0 && c->pending >= c->max_pending)) {
    hapod_status st = run_ready(c);
    if (st != HAPOD_OK) return st;
  }
  return HAPOD_OK;
}

hapod_status hapod_result(hapod_ctx* c, int64_t* k_out, double* sigma_host, void* dev_modes, int64_t ld_modes) {
  if (!c || !k_out) {
    if (c) c->err = "hapod_result: null k_out";
    g_thread_error = c ? "hapod_result: null k_out" : "hapod_result: null context";
    return HAPOD_ERR_INVALID;
  }
  if (c->poisoned) return HAPOD_ERR_STATE;
  if (c->leaves_pushed != c->leaves_total) {
    c->err = "hapod_result: not every leaf has been pushed";
    return HAPOD_ERR_STATE;
  }
  hapod_status st = run_ready(c);
  if (st != HAPOD_OK) return st;
  NodeRT& R = c->nodes[c->root];
  if (R.state != 2) {
    c->err = "hapod_result: root not finished";
    return HAPOD_ERR_STATE;
  }
  *k_out = R.k;
  if (dev_modes && R.k > 0) {
    if (ld_modes < c->n) {
      c->err = "hapod_result: ld_modes < n";
      return HAPOD_ERR_INVALID;
    }
    const size_t col_bytes = (size_t)c->n * c->esize;
    if (!c->env.cuda(cudaMemcpy2DAsync(dev_modes, (size_t)ld_modes * c->esize, c->result, (size_t)c->ldn * c->esize,
                                       col_bytes,
                                       (size_t)R.k, cudaMemcpyDeviceToDevice, c->env.s),
                     "copy result"))
      return ctx_fail(c);
  }
  if (sigma_host && R.k > 0) memcpy(sigma_host, R.sigma.data(), sizeof(double) * R.k);
  if (!c->env.cuda(cudaStreamSynchronize(c->env.s), "synchronize")) return ctx_fail(c);
  if (c->prof) c->prof->resolve();
  return c->warning;
}

hapod_status hapod_profile(hapod_ctx* c, hapod_profile_info* info) {
  if (!c || !info) {
    g_thread_error = c ? "hapod_profile: null info" : "hapod_profile: null context";
    return HAPOD_ERR_INVALID;
  }
  memset(info, 0, sizeof(*info));
  if (!c->prof) return HAPOD_OK;
  if (!c->env.cuda(cudaStreamSynchronize(c->env.s), "synchronize")) return ctx_fail(c);
  c->prof->resolve();
  *info = c->prof->acc;
  return HAPOD_OK;
}

hapod_status hapod_node_stats(const hapod_ctx* c, int32_t node, hapod_node_info* info) {
  if (!c || !info || node < 0 || node >= (int)c->nodes.size()) {
    g_thread_error = !c ? "hapod_node_stats: null context"
                        : !info ? "hapod_node_stats: null info" : "hapod_node_stats: node index out of range";
    return HAPOD_ERR_INVALID;
  }
  const NodeRT& A = c->nodes[node];
  info->m = A.state == 2 ? A.m : 0;
  info->k = A.state == 2 ? A.k : -1;
  info->eps = A.eps;
  info->tail_sq = A.tail;
  info->level = A.level;
  info->sweeps = A.sweeps;
  info->state = A.state;
  info->status = A.status;
  return HAPOD_OK;
}

const char* hapod_last_error(const hapod_ctx* c) { return c ? c->err.c_str() : g_thread_error.c_str(); }

void hapod_destroy(hapod_ctx* c) {
  if (!c) return;
  Env& env = c->env;
  for (NodeRT& A : c->nodes) {
    if (A.in_owned) env.release(A.in_owned);
    if (A.pbuf) env.release(A.pbuf);
    if (A.stash) env.release(A.stash);
    if (A.rv) env.release(A.rv);
  }
  env.release(c->result);
  cudaStreamSynchronize(env.s);
  if (c->stage.base) cudaFreeHost(c->stage.base);
  delete c->prof;
  delete c;
}

hapod_status hapod_result_right(hapod_ctx* c, double* W, int64_t ldw) {
  if (!c) {
    g_thread_error = "hapod_result_right: null context";
    return HAPOD_ERR_INVALID;
  }
  if (c->poisoned) return HAPOD_ERR_STATE;
  if (!c->keep_rv) {
    c->err = "hapod_result_right: context created without HAPOD_FLAG_RIGHT_VECTORS";
    return HAPOD_ERR_STATE;
  }
  NodeRT& R = c->nodes[c->root];
  if (R.state != 2) {
    c->err = "hapod_result_right: root not finished (call hapod_result first)";
    return HAPOD_ERR_STATE;
  }
  const int64_t k = std::max<int64_t>(0, R.k);
  if (k == 0) return HAPOD_OK;
  if (!W || ldw < c->S) {
    c->err = "hapod_result_right: null W or ldw < |S|";
    return HAPOD_ERR_INVALID;
  }
  Env& env = c->env;
  const int N = (int)c->nodes.size();
  // row offset of every leaf in the enumeration of S (leaves in node order)
  std::vector<int64_t> leaf_off(N, -1);
  int64_t off = 0;
  for (int a = 0; a < N; ++a)
    if (c->nodes[a].children.empty()) {
      leaf_off[a] = off;
      off += c->nodes[a].leaf_cols;
    }
  if (!env.cuda(cudaMemset2DAsync(W, (size_t)ldw * sizeof(double), 0, (size_t)c->S * sizeof(double), (size_t)k,
                                  env.s),
                "clear W"))
    return ctx_fail(c);
  // T_a (m_a x k): rows of Lambda~ below node a, mapped through a's input; the root's
  // is its own V_N.  Top-down: T_c = V_c T_a[pcol_c : pcol_c + k_c, :].
  std::vector<double*> T(N, nullptr);
  std::vector<int64_t> ldT(N, 0);
  std::vector<int> order{c->root};
  bool ok = true;
  auto place = [&](int a, const double* rows, int64_t ld_rows) -> bool {
    // a's map T_a = V_a rows (V_a = identity at pass-through nodes); leaves go to W
    NodeRT& A = c->nodes[a];
    double* dst;
    int64_t ldd;
    if (A.children.empty()) {
      dst = W + leaf_off[a];
      ldd = ldw;
    } else {
      T[a] = (double*)env.alloc(sizeof(double) * (size_t)A.m * (size_t)k, "alloc right-vector map");
      if (!T[a]) return false;
      ldT[a] = A.m;
      dst = T[a];
      ldd = A.m;
    }
    if (A.rv)
      return env.cuda(launch_gemm_nn_f64(A.m, k, A.k, A.rv, A.m, rows, ld_rows, dst, ldd, env.s), "right-vector product");
    return env.cuda(cudaMemcpy2DAsync(dst, (size_t)ldd * sizeof(double), rows, (size_t)ld_rows * sizeof(double),
                                      (size_t)A.m * sizeof(double), (size_t)k, cudaMemcpyDeviceToDevice, env.s),
                    "copy right-vector rows");
  };
  // root: rows = identity (k x k)
  {
    std::vector<double> eye((size_t)k * k, 0.0);
    for (int64_t j = 0; j < k; ++j) eye[(size_t)j * k + j] = 1.0;
    double* eye_d = env.upload(eye, "upload identity");
    ok = eye_d && place(c->root, eye_d, k);
    ok = ok && env.cuda(cudaStreamSynchronize(env.s), "synchronize");
    env.release(eye_d);
  }
  for (size_t h = 0; h < order.size() && ok; ++h) {
    const int a = order[h];
    for (int ch : c->nodes[a].children) {
      NodeRT& C = c->nodes[ch];
      if (C.k <= 0) continue;  // no modes reached the parent: its rows of W stay zero
      if (C.pcol < 0) {
        c->err = "hapod_result_right: a child's position in its parent's input is unknown";
        ok = false;
        break;
      }
      ok = place(ch, T[a] + C.pcol, ldT[a]);
      if (!C.children.empty()) order.push_back(ch);
      if (!ok) break;
    }
  }
  ok = ok && env.cuda(cudaStreamSynchronize(env.s), "synchronize");
  for (double* t : T) env.release(t);
  if (!ok) {
    if (c->err == "no error" || c->err.empty()) c->err = env.err;
    return env.code != HAPOD_OK ? ctx_fail(c) : HAPOD_ERR_STATE;
  }
  return HAPOD_OK;
}

hapod_status hapod_trim_pool(void* stream) {
  Env env;
  if (!init_env(env, stream)) {
    g_thread_error = env.err;
    return env.code;
  }
  if (!env.cuda(cudaStreamSynchronize(env.s), "synchronize") ||
      !env.cuda(cudaMemPoolTrimTo(env.pool, 0), "cudaMemPoolTrimTo")) {
    g_thread_error = env.err;
    return env.code;
  }
  return HAPOD_OK;
}

// ------------------------------------------------------------- single-node steps
static hapod_status step_error(Env& env) {
  g_thread_error = env.err;
  return env.code;
}

hapod_status hapod_gram(int32_t precision, int64_t n, int64_t m, const void* X, int64_t ldx, double* G,
                        void* stream) {
  if (!valid_precision(precision) || n < 0 || m < 0 || ldx < n || (m > 0 && (!X || !G)) || m > INT32_MAX) {
    g_thread_error = "hapod_gram: invalid argument";
    return HAPOD_ERR_INVALID;
  }
  if (m == 0) return HAPOD_OK;
  Env env;
  if (!init_env(env, stream)) return step_error(env);
  if (n == 0) {
    if (!env.cuda(cudaMemsetAsync(G, 0, sizeof(double) * m * m, env.s), "memset")) return step_error(env);
    return HAPOD_OK;
  }
  Work w;
  w.X = X;
  w.ldx = ldx;
  w.n = n;
  w.m = m;
  w.G = G;
  std::vector<Work*> ws{&w};
  if (precision == HAPOD_FP64) {
    if (!step_gram(env, precision, ws)) return step_error(env);
    return HAPOD_OK;
  }
  // tensor-core forms: aligned input for TMA (mixed form), device error flag read back here
  bool ok = true;
  if (mixed_form(precision) && !tma_compatible_f32(X, ldx)) {
    const int64_t ld = (n + 31) / 32 * 32;
    w.X_tmp = env.alloc(sizeof(float) * ld * m, "alloc aligned input");
    ok = w.X_tmp && env.cuda(cudaMemcpy2DAsync(w.X_tmp, ld * sizeof(float), X, ldx * sizeof(float),
                                               n * sizeof(float), m, cudaMemcpyDeviceToDevice, env.s),
                             "copy input for TMA");
    w.X = w.X_tmp;
    w.ldx = ld;
  }
  env.err_dev = ok ? (int*)env.alloc(sizeof(int) * 2, "alloc flag") : nullptr;
  ok = ok && env.err_dev && env.cuda(cudaMemsetAsync(env.err_dev, 0, sizeof(int) * 2, env.s), "memset") &&
       init_err_flag(env, env.err_dev) && step_gram(env, precision, ws);
  int dev_err = 0;
  if (ok) ok = env.cuda(cudaMemcpyAsync(&dev_err, env.err_dev, sizeof(int), cudaMemcpyDeviceToHost, env.s), "read flag");
  env.release(env.err_dev);
  env.release(w.X_tmp);
  env.release(w.exps);
  ok = env.cuda(cudaStreamSynchronize(env.s), "synchronize") && ok;
  if (!ok) return step_error(env);
  if (dev_err) {
    g_thread_error = "hapod_gram: device-side wait timed out";
    return HAPOD_ERR_TIMEOUT;
  }
  return HAPOD_OK;
}

hapod_status hapod_eig(int32_t precision, int64_t m, const double* G, double* lambda, double* V, int32_t* sweeps_host,
                       void* stream) {
  if (!valid_precision(precision) || m < 0 || m > INT32_MAX || (m > 0 && (!G || !lambda || !V))) {
    g_thread_error = "hapod_eig: invalid argument";
    return HAPOD_ERR_INVALID;
  }
  if (m > kEigMaxM) {  // checked on the host before any CUDA call, like the other arguments
    g_thread_error = "hapod_eig: node wider than the eigensolver supports (13000 columns)";
    return HAPOD_ERR_INVALID;
  }
  if (sweeps_host) *sweeps_host = 0;
  if (m == 0) return HAPOD_OK;
  Env env;
  if (!init_env(env, stream)) return step_error(env);
  const bool vf64 = eigvec_f64(precision);
  Work w;
  w.m = m;
  std::vector<Work*> ws{&w};
  if (!alloc_work(env, ws, vf64)) {
    free_work(env, ws);
    return step_error(env);
  }
  NodeResult* res_d = (NodeResult*)env.alloc(sizeof(NodeResult), "alloc result");
  bool ok = res_d && env.cuda(cudaMemsetAsync(res_d, 0, sizeof(NodeResult), env.s), "memset") &&
            env.cuda(cudaMemcpyAsync(w.G, G, sizeof(double) * m * m, cudaMemcpyDeviceToDevice, env.s), "copy G") &&
            step_eig(env, precision, ws, res_d);
  if (ok) {
    GatherJob g;
    g.V = w.V;
    g.perm = w.perm;
    g.Vk = V;
    g.m = (int32_t)m;
    g.k = (int32_t)m;
    std::vector<GatherJob> gj{g};
    GatherJob* gd = env.upload(gj, "upload gather");
    ok = gd && env.cuda(launch_gather(vf64, gd, 1, env.s), "gather launch") &&
         env.cuda(cudaMemcpyAsync(lambda, w.lambda, sizeof(double) * m, cudaMemcpyDeviceToDevice, env.s), "copy");
    env.release(gd);
  }
  NodeResult r{};
  if (ok) ok = env.cuda(cudaMemcpyAsync(&r, res_d, sizeof(r), cudaMemcpyDeviceToHost, env.s), "read back");
  env.release(res_d);
  free_work(env, ws);
  ok = env.cuda(cudaStreamSynchronize(env.s), "synchronize") && ok;
  if (!ok) return step_error(env);
  if (sweeps_host) *sweeps_host = r.sweeps;
  if (r.status != HAPOD_OK) g_thread_error = "hapod_eig: see status";
  return (hapod_status)r.status;
}

hapod_status hapod_truncate(int64_t m, const double* lambda, double eps, int64_t* N_host, double* tail_host,
                            void* stream) {
  if (m < 0 || m > INT32_MAX || !(eps >= 0.0) || !N_host || (m > 0 && eps > 0.0 && !lambda)) {
    g_thread_error = "hapod_truncate: invalid argument";
    return HAPOD_ERR_INVALID;
  }
  if (eps == 0.0 || m == 0) {
    *N_host = m;
    if (tail_host) *tail_host = 0.0;
    return HAPOD_OK;
  }
  Env env;
  if (!init_env(env, stream)) return step_error(env);
  Work w;
  w.m = m;
  w.eps = eps;
  w.lambda = const_cast<double*>(lambda);
  w.sigma = (double*)env.alloc(sizeof(double) * m, "alloc sigma");
  NodeResult* res_d = (NodeResult*)env.alloc(sizeof(NodeResult), "alloc result");
  std::vector<Work*> ws{&w};
  NodeResult r{};
  bool ok = w.sigma && res_d && env.cuda(cudaMemsetAsync(res_d, 0, sizeof(NodeResult), env.s), "memset") &&
            step_truncate(env, ws, res_d) &&
            env.cuda(cudaMemcpyAsync(&r, res_d, sizeof(r), cudaMemcpyDeviceToHost, env.s), "read back");
  env.release(w.sigma);
  env.release(res_d);
  ok = env.cuda(cudaStreamSynchronize(env.s), "synchronize") && ok;
  if (!ok) return step_error(env);
  *N_host = r.k;
  if (tail_host) *tail_host = r.tail;
  return HAPOD_OK;
}

hapod_status hapod_modes(int32_t precision, int64_t n, int64_t m, const void* X, int64_t ldx, const double* V,
                         int64_t ldv, int64_t N, const double* scale, void* Y, int64_t ldy, void* stream) {
  if (!valid_precision(precision) || n < 0 || m < 0 || N < 0 || N > m || ldx < n || ldv < m || ldy < n ||
      m > INT32_MAX || (N > 0 && n > 0 && (!X || !V || !Y))) {
    g_thread_error = "hapod_modes: invalid argument";
    return HAPOD_ERR_INVALID;
  }
  if (N == 0 || n == 0) return HAPOD_OK;
  Env env;
  if (!init_env(env, stream)) return step_error(env);
  if (precision == HAPOD_FP64_OZAKI || precision == HAPOD_MIXED_FX3) {
    // tensor-core kernel with bounded waits: its error flag is read back here
    Work w;
    w.X = X;
    w.ldx = ldx;
    if (precision == HAPOD_MIXED_FX3 && !tma_compatible_f32(X, ldx)) {  // TMA: aligned copy
      const int64_t ld = (n + 31) / 32 * 32;
      w.X_tmp = env.alloc(sizeof(float) * ld * m, "alloc aligned input");
      if (!w.X_tmp || !env.cuda(cudaMemcpy2DAsync(w.X_tmp, ld * sizeof(float), X, ldx * sizeof(float),
                                                  n * sizeof(float), m, cudaMemcpyDeviceToDevice, env.s),
                                "copy input for TMA"))
        return step_error(env);
      w.X = w.X_tmp;
      w.ldx = ld;
    }
    w.n = n;
    w.m = m;
    w.Vk = const_cast<double*>(V);
    w.ldvk = ldv;
    w.scale = const_cast<double*>(scale);
    w.Y = Y;
    w.ldy = ldy;
    w.res.k = (int32_t)N;
    std::vector<Work*> ws{&w};
    env.err_dev = (int*)env.alloc(sizeof(int) * 2, "alloc flag");
    bool ok = env.err_dev && env.cuda(cudaMemsetAsync(env.err_dev, 0, sizeof(int) * 2, env.s), "memset") &&
              init_err_flag(env, env.err_dev) &&
              (precision == HAPOD_FP64_OZAKI ? step_modes_oz(env, ws) : step_modes_fx(env, ws));
    int dev_err = 0;
    if (ok)
      ok = env.cuda(cudaMemcpyAsync(&dev_err, env.err_dev, sizeof(int), cudaMemcpyDeviceToHost, env.s), "read flag");
    env.release(env.err_dev);
    env.release(w.exps);
    env.release(w.X_tmp);
    ok = env.cuda(cudaStreamSynchronize(env.s), "synchronize") && ok;
    if (!ok) return step_error(env);
    if (dev_err) {
      g_thread_error = "hapod_modes: device-side wait timed out";
      return HAPOD_ERR_TIMEOUT;
    }
    return HAPOD_OK;
  }
  const bool fp64 = f64_data(precision);
  const int tr = fp64 ? modes_f64_tile_rows((int)N) : modes_mixed_rows_per_block((int)N);
  const int tc = fp64 ? modes_f64_tile_cols((int)N) : modes_mixed_tile_cols((int)N);
  ModesJob J;
  memset(&J, 0, sizeof(J));
  J.X = X;
  J.ldx = ldx;
  J.Vk = V;
  J.ldv = ldv;
  J.scale = scale;
  J.Y = Y;
  J.ldy = ldy;
  J.n = n;
  J.m = (int32_t)m;
  J.k = (int32_t)N;
  J.row_tiles = (int32_t)((n + tr - 1) / tr);
  J.col_tiles = (int32_t)((N + tc - 1) / tc);
  J.block_base = 0;
  std::vector<ModesJob> mj{J};
  ModesJob* md = env.upload(mj, "upload modes job");
  if (!md) return step_error(env);
  const int64_t blocks = (int64_t)J.row_tiles * J.col_tiles;
  bool ok;
  if (fp64)
    ok = env.cuda(launch_modes_f64(md, 1, blocks, tc, env.s), "modes launch");
  else
    ok = env.cuda(launch_modes_mixed(md, 1, blocks, tc, tma_compatible_f32(X, ldx) && tma_compatible_f32(Y, ldy), env.s),
                  "modes launch");
  env.release(md);
  if (!ok) return step_error(env);
  return HAPOD_OK;
}

hapod_status hapod_pod(int32_t precision, int64_t n, int64_t m, const void* X, int64_t ldx, double eps,
                       int64_t* N_host, double* sigma, void* Y, int64_t ldy, double* tail_host, void* stream) {
  if (!valid_precision(precision) || n < 1 || m < 0 || m > INT32_MAX || ldx < n || ldy < n || !(eps >= 0.0) ||
      !N_host || (m > 0 && (!X || !Y || !sigma))) {
    g_thread_error = "hapod_pod: invalid argument";
    return HAPOD_ERR_INVALID;
  }
  if (eps > 0.0 && m > kEigMaxM) {
    g_thread_error = "hapod_pod: node wider than the eigensolver supports (13000 columns)";
    return HAPOD_ERR_INVALID;
  }
  Env env;
  if (!init_env(env, stream)) return step_error(env);
  const size_t es = elem_size(precision);
  if (eps == 0.0 || m == 0) {  // POD(S, 0) = {(1, s)}
    *N_host = m;
    if (tail_host) *tail_host = 0.0;
    if (m == 0) return HAPOD_OK;
    std::vector<double> ones((size_t)m, 1.0);
    bool ok = env.cuda(cudaMemcpyAsync(sigma, ones.data(), sizeof(double) * m, cudaMemcpyHostToDevice, env.s), "copy") &&
              env.cuda(cudaMemcpy2DAsync(Y, ldy * es, X, ldx * es, n * es, m, cudaMemcpyDeviceToDevice, env.s),
                       "copy") &&
              env.cuda(cudaStreamSynchronize(env.s), "synchronize");
    return ok ? HAPOD_OK : step_error(env);
  }
  Work w;
  w.X = X;
  w.ldx = ldx;
  w.n = n;
  w.m = m;
  w.eps = eps;
  std::vector<Work*> ws{&w};
  bool ok = run_pod_front(env, precision, ws);
  if (ok && w.res.k > 0) {
    w.Y = Y;
    w.ldy = ldy;
    ok = env.cuda(cudaMemcpyAsync(sigma, w.sigma, sizeof(double) * w.res.k, cudaMemcpyDeviceToDevice, env.s),
                  "copy sigma") &&
         run_pod_back(env, precision, ws);
  }
  free_work(env, ws);
  ok = env.cuda(cudaStreamSynchronize(env.s), "synchronize") && ok;
  if (!ok) return step_error(env);
  *N_host = w.res.k;
  if (tail_host) *tail_host = w.res.tail;
  return (hapod_status)(w.res.status >= HAPOD_WARN_NOCONVERGE ? w.res.status : HAPOD_OK);
}

hapod_status hapod_autotune(int32_t precision, int64_t n, int64_t m, const void* X, int64_t ldx, int32_t* pct_out,
                            double* ms_out, void* stream) {
  if (!(precision == HAPOD_FP64 || precision == HAPOD_MIXED_TF32X3 || precision == HAPOD_MIXED_BF16X3 ||
        precision == HAPOD_MIXED_FX3) ||
      n < 1 || m < 1 || m > kEigMaxM || !X || ldx < n) {
    g_thread_error = "hapod_autotune: invalid argument (forms FP64, TF32X3, BF16X3, FX3; n, m >= 1, ld >= n)";
    return HAPOD_ERR_INVALID;
  }
  static const int kCand[4] = {50, 100, 200, 400};
  const auto key = std::make_tuple((int)precision, log2_bucket(m), log2_bucket(n));
  Env env;
  if (!init_env(env, stream)) return step_error(env);
  double* G = (double*)env.alloc(sizeof(double) * (size_t)m * (size_t)m, "alloc Gram");
  if (!G) return step_error(env);
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  bool ok = env.cuda(cudaEventCreate(&e0), "event") && env.cuda(cudaEventCreate(&e1), "event");
  double best = 1e300;
  int best_pct = 100;
  hapod_status st = HAPOD_OK;
  for (int c = 0; c < 4 && ok; ++c) {
    {
      std::lock_guard<std::mutex> lk(g_tune_mu);
      g_tune[key] = kCand[c];
    }
    st = hapod_gram(precision, n, m, X, ldx, G, stream);  // warm-up (and correctness of the plan)
    float tot = 0.f;
    for (int r = 0; r < 3 && st == HAPOD_OK && ok; ++r) {
      ok = env.cuda(cudaEventRecord(e0, env.s), "event record");
      st = hapod_gram(precision, n, m, X, ldx, G, stream);
      float ms = 0.f;
      ok = ok && env.cuda(cudaEventRecord(e1, env.s), "event record") &&
           env.cuda(cudaEventSynchronize(e1), "event sync") && env.cuda(cudaEventElapsedTime(&ms, e0, e1), "elapsed");
      tot += ms;
    }
    if (st != HAPOD_OK) break;
    const double ms = tot / 3.0;
    if (ms_out) ms_out[c] = ms;
    if (ms < best * 0.98) {  // a new factor has to win by 2 %
      best = ms;
      best_pct = kCand[c];
    }
  }
  {
    std::lock_guard<std::mutex> lk(g_tune_mu);
    if (ok && st == HAPOD_OK) g_tune[key] = best_pct;
    else g_tune.erase(key);
  }
  if (e0) cudaEventDestroy(e0);
  if (e1) cudaEventDestroy(e1);
  env.release(G);
  cudaStreamSynchronize(env.s);
  if (st != HAPOD_OK) return st;
  if (!ok) return step_error(env);
  if (pct_out) *pct_out = best_pct;
  return HAPOD_OK;
}

void hapod_autotune_clear(void) {
  std::lock_guard<std::mutex> lk(g_tune_mu);
  g_tune.clear();
}

}  // extern "C"
