// Batching form: uneven batches of states evaluated by persistent kernels,
// replayable as a captured CUDA graph, with a launch shape chosen by an
// autotuner (threads per block, resident blocks per SM, per-state arrays in
// shared memory or in a global workspace).
//
// A plan owns device copies of the batch descriptors, a per-group tile
// table and work counter, and the workspace.  Batches are split into groups
// ("waves") of at most max_states_per_launch states; each group is one
// persistent launch in which warps take 32-state tiles from an atomic counter
// until the group's tiles run out (no waiting, so no wait needs a bound).
// Batches of different groups may share output memory.
#include <cuda_runtime.h>

#include <algorithm>
#include <cstdio>
#include <cstring>
#include <fstream>
#include <map>
#include <mutex>
#include <sstream>
#include <string>
#include <vector>

#include "kinetics_state.cuh"
#include "launch.h"


struct pj_plan {
  const pj_mech* mech = nullptr;
  int op = 0, mode = 0, fmt = 0, nb = 0;
  int* d_status = nullptr;
  std::vector<pj_batch> batches;
  struct Group {
    std::vector<int> idx;
    int64_t tiles = 0;
    void* d_batches = nullptr;      // BatchDev[]
    int64_t* d_tile_start = nullptr;
    unsigned long long* d_counter = nullptr;
  };
  std::vector<Group> groups;
  int tpb = 128, bps = 1, use_smem = 1;
  pj::CoopPlan coop{};  // tpb 256 / 512: the cooperative Jacobian kernel
  int grid = 0;
  size_t smem = 0;
  double* ws = nullptr;
  size_t ws_bytes = 0;
  cudaGraph_t graph = nullptr;
  cudaGraphExec_t exec = nullptr;
};

namespace pj {

using BatchDev = CoopBatch;  // (param, phi, out, dphi, n, ld) of one batch

// Persistent kernel: OP 0 = source terms, 1 = analytical Jacobian (FP64).
template <int OP, int MODE, int FMT, bool SPECIAL>
__global__ void __launch_bounds__(128, 4) k_batched(DevMech m, const BatchDev* __restrict__ batches,
                                                    const int64_t* __restrict__ tile_start, int nb,
                                                    unsigned long long* counter, int* status, double* ws,
                                                    int64_t ws_stride) {
  PJ_DYN_SMEM;
  load_exp_table(m.exp_tab);
  const int64_t gtid = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  const int lane = threadIdx.x & 31;
  StateArrays A;
  A.ns = m.ns;
  if (ws) {
    A.base = ws + gtid;
    A.stride = ws_stride;
  } else {
    A.base = smem + threadIdx.x;
    A.stride = blockDim.x;
  }
  const int64_t total = tile_start[nb];
  for (;;) {
    unsigned long long t = 0;
    if (lane == 0) t = atomicAdd(counter, 1ULL);
    const int64_t tile = (int64_t)__shfl_sync(0xffffffffu, t, 0);
    if (tile >= total) break;
    // the batch holding this tile: the largest b with tile_start[b] <= tile
    int lo = 0, hi = nb - 1;
    while (lo < hi) {
      const int mid = (lo + hi + 1) >> 1;
      if (__ldg(tile_start + mid) <= tile) lo = mid;
      else hi = mid - 1;
    }
    const BatchDev B = batches[lo];
    const int64_t s = (tile - __ldg(tile_start + lo)) * 32 + lane;
    if (s < B.n) {
      if (OP == 0)
        source_state<MODE, SPECIAL>(m, A, B.param, B.phi, B.ld, s, B.out, status);
      else
        jacobian_state<MODE, FMT, double, false, false, SPECIAL>(m, A, B.param, B.phi, B.ld, s, B.out, B.dphi,
                                                                 status, nullptr, 0.0);
    }
  }
}

template <int OP, int MODE, int FMT>
static int launch_group(const pj_plan* p, const pj_plan::Group& g, cudaStream_t st) {
  if (p->coop.use) {
    // the cooperative kernel (a 32-state tile per block) over the group's
    // tiles, handed out by the same counter
    cudaError_t e = cudaMemsetAsync(g.d_counter, 0, sizeof(unsigned long long), st);
    if (e != cudaSuccess) return check_cuda(e, "cudaMemsetAsync(plan counter)");
    JacArgs a{nullptr, nullptr, 0, nullptr, nullptr, p->d_status, nullptr, 0.0,
              CoopSrc{static_cast<const CoopBatch*>(g.d_batches), g.d_tile_start, (int)g.idx.size(), g.d_counter}};
    return launch_jac_coop_f64(p->mech->dm, p->coop, MODE, FMT, g.tiles * 32, a, p->ws, st);
  }
  auto kern = p->mech->dm.nr_plain < p->mech->dm.nr ? k_batched<OP, MODE, FMT, true> : k_batched<OP, MODE, FMT, false>;
  cudaError_t e = cudaMemsetAsync(g.d_counter, 0, sizeof(unsigned long long), st);
  if (e != cudaSuccess) return check_cuda(e, "cudaMemsetAsync(plan counter)");
  kern<<<p->grid, p->tpb, p->smem, st>>>(p->mech->dm, static_cast<const BatchDev*>(g.d_batches), g.d_tile_start,
                                         (int)g.idx.size(), g.d_counter, p->d_status, p->use_smem ? nullptr : p->ws,
                                         (int64_t)p->grid * p->tpb);
  return check_cuda(cudaGetLastError(), "k_batched launch");
}

template <int OP, int MODE, int FMT>
static int set_kernel_smem(const DevMech& m, size_t smem) {
  if (m.nr_plain < m.nr) return set_smem(k_batched<OP, MODE, FMT, true>, smem);
  return set_smem(k_batched<OP, MODE, FMT, false>, smem);
}

// dispatch over (op, mode, fmt)
template <typename F>
static int dispatch(int op, int mode, int fmt, F&& f) {
  if (op == 0) {
    if (mode == PJ_CONP) return f.template go<0, PJ_CONP, PJ_CSR>();
    return f.template go<0, PJ_CONV, PJ_CSR>();
  }
  if (mode == PJ_CONP) {
    if (fmt == PJ_CSR) return f.template go<1, PJ_CONP, PJ_CSR>();
    if (fmt == PJ_CSC) return f.template go<1, PJ_CONP, PJ_CSC>();
    return f.template go<1, PJ_CONP, PJ_DENSE>();
  }
  if (fmt == PJ_CSR) return f.template go<1, PJ_CONV, PJ_CSR>();
  if (fmt == PJ_CSC) return f.template go<1, PJ_CONV, PJ_CSC>();
  return f.template go<1, PJ_CONV, PJ_DENSE>();
}

struct RunGroups {
  const pj_plan* p;
  cudaStream_t st;
  template <int OP, int MODE, int FMT>
  int go() {
    for (const auto& g : p->groups) {
      if (g.tiles == 0) continue;
      int rc = launch_group<OP, MODE, FMT>(p, g, st);
      if (rc) return rc;
    }
    return PJ_OK;
  }
};

struct SetSmem {
  const DevMech& m;
  size_t smem;
  template <int OP, int MODE, int FMT>
  int go() { return set_kernel_smem<OP, MODE, FMT>(m, smem); }
};

static int plan_arrays(const pj_plan* p) { return p->op == 0 ? source_arrays() : jacobian_arrays(); }

static void drop_graph(pj_plan* p) {
  if (p->exec) cudaGraphExecDestroy(p->exec);
  if (p->graph) cudaGraphDestroy(p->graph);
  p->exec = nullptr;
  p->graph = nullptr;
}

// Apply a launch shape: grid, shared memory or workspace (reallocated when it
// must grow).
static int64_t plan_max_tiles(const pj_plan* p) {
  int64_t t = 0;
  for (const auto& g : p->groups) t = std::max(t, g.tiles);
  return t;
}

// workspace of at least `need` bytes (reallocated when it must grow)
static int plan_workspace(pj_plan* p, size_t need) {
  if (need <= p->ws_bytes) return PJ_OK;
  if (p->ws) cudaFree(p->ws);
  p->ws = nullptr;
  p->ws_bytes = 0;
  cudaError_t e = cudaMalloc(&p->ws, need);
  if (e != cudaSuccess) return check_cuda(e, "cudaMalloc(plan workspace)");
  p->ws_bytes = need;
  return PJ_OK;
}

static int plan_configure(pj_plan* p, int tpb, int bps, int use_smem) {
  if (tpb == 256 || tpb == 512) {
    // cooperative: tpb / 32 warps share each 32-state tile
    if (p->op != 1) return fail(PJ_ERR_UNSUPPORTED, "plan: the cooperative layout computes Jacobians only");
    CoopPlan c{};
    if (!coop_shape(p->mech->dm, tpb / 32, bps, use_smem != 0, plan_max_tiles(p), c))
      return fail(PJ_ERR_UNSUPPORTED, "plan: cooperative shape does not fit (blocks x warps <= 16 per SM, "
                                      "shared memory)");
    drop_graph(p);
    int rc = plan_workspace(p, c.ws_bytes);
    if (rc) return rc;
    p->tpb = tpb;
    p->bps = bps;
    p->use_smem = use_smem ? 1 : 0;
    p->coop = c;
    p->grid = c.grid;
    p->smem = c.smem;
    return PJ_OK;
  }
  if (tpb != 32 && tpb != 64 && tpb != 128)
    return fail(PJ_ERR_ARG, "plan: threads per block must be 32, 64 or 128 (256 or 512: cooperative)");
  if (bps < 1 || bps > 16) return fail(PJ_ERR_ARG, "plan: blocks per SM must be 1..16");
  const size_t per_thread = (size_t)plan_arrays(p) * p->mech->ns * sizeof(double);
  const size_t smem_cap = 225 * 1024;
  if (use_smem && per_thread * tpb > smem_cap)
    return fail(PJ_ERR_UNSUPPORTED, "plan: per-state arrays do not fit shared memory at this block size");
  drop_graph(p);
  p->tpb = tpb;
  p->bps = bps;
  p->use_smem = use_smem;
  p->coop = CoopPlan{};
  p->grid = sm_count() * bps;
  p->smem = use_smem ? per_thread * tpb : 0;
  if (use_smem) return dispatch(p->op, p->mode, p->fmt, SetSmem{p->mech->dm, p->smem});
  return plan_workspace(p, per_thread * (size_t)p->grid * tpb);
}

static void plan_release(pj_plan* p) {
  drop_graph(p);
  for (auto& g : p->groups) {
    if (g.d_batches) cudaFree(g.d_batches);
    if (g.d_tile_start) cudaFree(g.d_tile_start);
    if (g.d_counter) cudaFree(g.d_counter);
  }
  if (p->ws) cudaFree(p->ws);
}

// ---- autotune cache: one JSON object per line, keyed by GPU, mechanism
// constants hash, op, mode and format
static std::mutex g_cache_mutex;

static uint64_t fnv1a(const void* data, size_t n, uint64_t h = 1469598103934665603ULL) {
  const unsigned char* b = static_cast<const unsigned char*>(data);
  for (size_t i = 0; i < n; i++) {
    h ^= b[i];
    h *= 1099511628211ULL;
  }
  return h;
}

static std::string plan_key(const pj_plan* p) {
  const pj_mech* m = p->mech;
  uint64_t h = fnv1a(m->W.data(), m->W.size() * sizeof(double));
  h = fnv1a(m->nasa_low.data(), m->nasa_low.size() * sizeof(double), h);
  h = fnv1a(m->A.data(), m->A.size() * sizeof(double), h);
  h = fnv1a(m->reac_sp.data(), m->reac_sp.size() * sizeof(int32_t), h);
  h = fnv1a(m->prod_sp.data(), m->prod_sp.size() * sizeof(int32_t), h);
  h = fnv1a(m->kind.data(), m->kind.size() * sizeof(int32_t), h);
  cudaDeviceProp prop{};
  int dev = 0;
  cudaGetDevice(&dev);
  cudaGetDeviceProperties(&prop, dev);
  char buf[512];
  snprintf(buf, sizeof buf, "%s|%016llx|ns%d|nr%d|op%d|mode%d|fmt%d", prop.name, (unsigned long long)h, m->ns, m->nr,
           p->op, p->mode, p->fmt);
  return buf;
}

static bool cache_lookup(const char* path, const std::string& key, int* tpb, int* bps, int* sm) {
  if (!path) return false;
  std::lock_guard<std::mutex> lk(g_cache_mutex);
  std::ifstream in(path);
  std::string line;
  bool found = false;
  while (std::getline(in, line)) {
    const std::string tag = "\"key\": \"" + key + "\"";
    if (line.find(tag) == std::string::npos) continue;
    int a, b, c;
    const size_t pos = line.find("\"tpb\":");
    if (pos != std::string::npos && sscanf(line.c_str() + pos, "\"tpb\": %d, \"bps\": %d, \"smem\": %d", &a, &b, &c) == 3) {
      *tpb = a;
      *bps = b;
      *sm = c;
      found = true;  // the last matching line wins
    }
  }
  return found;
}

static void cache_store(const char* path, const std::string& key, int tpb, int bps, int sm, double ms) {
  if (!path) return;
  std::lock_guard<std::mutex> lk(g_cache_mutex);
  std::ofstream out(path, std::ios::app);
  out << "{\"key\": \"" << key << "\", \"tpb\": " << tpb << ", \"bps\": " << bps << ", \"smem\": " << sm
      << ", \"ms\": " << ms << "}\n";
}

}  // namespace pj

using namespace pj;

extern "C" int pj_plan_create(const pj_mech* m, int op, int mode, int fmt, int n_batches, const pj_batch* batches,
                              int64_t max_states_per_launch, int* d_status, pj_plan** out) {
  if (!m || !out || (n_batches > 0 && !batches)) return fail(PJ_ERR_ARG, "pj_plan_create: null argument");
  *out = nullptr;
  if (op != PJ_OP_SOURCE && op != PJ_OP_JACOBIAN) return fail(PJ_ERR_ARG, "pj_plan_create: op must be PJ_OP_SOURCE or PJ_OP_JACOBIAN");
  if (mode != PJ_CONP && mode != PJ_CONV) return fail(PJ_ERR_ARG, "pj_plan_create: bad mode");
  if (op == PJ_OP_JACOBIAN && fmt != PJ_CSR && fmt != PJ_CSC && fmt != PJ_DENSE)
    return fail(PJ_ERR_ARG, "pj_plan_create: bad fmt");
  if (n_batches < 0 || max_states_per_launch < 0) return fail(PJ_ERR_ARG, "pj_plan_create: negative size");
  if (m->device < 0) return fail(PJ_ERR_CUDA, "pj_plan_create: mechanism has no device copy");
  int dev = -1;
  cudaGetDevice(&dev);
  if (dev != m->device) return fail(PJ_ERR_ARG, "pj_plan_create: current device differs from the mechanism's");
  for (int b = 0; b < n_batches; b++) {
    const pj_batch& B = batches[b];
    if (B.n < 0 || B.ld < B.n || B.ld < 1) return fail(PJ_ERR_ARG, "pj_plan_create: batch " + std::to_string(b) + ": bad n/ld");
    if (B.n > 0 && (!B.d_param || !B.d_phi || !B.d_out || (op == PJ_OP_JACOBIAN && !B.d_dphi)))
      return fail(PJ_ERR_ARG, "pj_plan_create: batch " + std::to_string(b) + ": null buffer");
  }
  pj_plan* p = new (std::nothrow) pj_plan();
  if (!p) return fail(PJ_ERR_NOMEM, "pj_plan_create: out of host memory");
  p->mech = m;
  p->op = op == PJ_OP_SOURCE ? 0 : 1;
  p->mode = mode;
  p->fmt = op == PJ_OP_JACOBIAN ? fmt : PJ_CSR;
  p->nb = n_batches;
  p->d_status = d_status;
  p->batches.assign(batches, batches + n_batches);
  // groups of consecutive batches, at most max_states_per_launch states each
  pj_plan::Group cur;
  int64_t cur_states = 0;
  for (int b = 0; b < n_batches; b++) {
    const int64_t nb_states = batches[b].n;
    if (!cur.idx.empty() && max_states_per_launch > 0 && cur_states + nb_states > max_states_per_launch) {
      p->groups.push_back(cur);
      cur = pj_plan::Group();
      cur_states = 0;
    }
    cur.idx.push_back(b);
    cur_states += nb_states;
  }
  if (!cur.idx.empty()) p->groups.push_back(cur);
  int rc = PJ_OK;
  for (auto& g : p->groups) {
    std::vector<BatchDev> bd;
    std::vector<int64_t> ts(1, 0);
    for (int b : g.idx) {
      const pj_batch& B = batches[b];
      bd.push_back(BatchDev{B.d_param, B.d_phi, B.d_out, B.d_dphi, B.n, B.ld});
      ts.push_back(ts.back() + (B.n + 31) / 32);
    }
    g.tiles = ts.back();
    cudaError_t e = cudaMalloc(&g.d_batches, bd.size() * sizeof(BatchDev));
    if (e == cudaSuccess) e = cudaMalloc(&g.d_tile_start, ts.size() * sizeof(int64_t));
    if (e == cudaSuccess) e = cudaMalloc(&g.d_counter, sizeof(unsigned long long));
    if (e == cudaSuccess) e = cudaMemcpy(g.d_batches, bd.data(), bd.size() * sizeof(BatchDev), cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMemcpy(g.d_tile_start, ts.data(), ts.size() * sizeof(int64_t), cudaMemcpyHostToDevice);
    if (e != cudaSuccess) {
      rc = check_cuda(e, "pj_plan_create: device tables");
      break;
    }
  }
  if (!rc) {
    // default shape: shared memory when 128 threads' arrays fit; else, for
    // the Jacobian, the cooperative layout (16 warps a block, arrays in
    // shared memory where they fit, else in the workspace: one 32-state tile
    // per SM keeps them in L2), for source terms a global workspace with 4
    // resident blocks of 128 per SM
    const size_t per_thread = (size_t)plan_arrays(p) * m->ns * sizeof(double);
    const int fit = (int)((225 * 1024 / per_thread) / 32 * 32);
    if (fit >= 128) rc = plan_configure(p, fit >= 256 ? 128 : (fit % 64 == 0 ? 64 : 32), 1, 1);
    else if (p->op == 1) {
      rc = plan_configure(p, 512, 1, 1);
      if (rc == PJ_ERR_UNSUPPORTED) rc = plan_configure(p, 512, 1, 0);
    } else rc = plan_configure(p, 128, 4, 0);
  }
  if (rc) {
    plan_release(p);
    delete p;
    return rc;
  }
  *out = p;
  return PJ_OK;
}

extern "C" int pj_plan_free(pj_plan* p) {
  if (!p) return PJ_OK;
  plan_release(p);
  delete p;
  return PJ_OK;
}

extern "C" int pj_plan_set_config(pj_plan* p, int threads_per_block, int blocks_per_sm, int use_shared) {
  if (!p) return fail(PJ_ERR_ARG, "pj_plan_set_config: null plan");
  return plan_configure(p, threads_per_block, blocks_per_sm, use_shared ? 1 : 0);
}

extern "C" int pj_plan_get_config(const pj_plan* p, int* threads_per_block, int* blocks_per_sm, int* use_shared,
                                  int* n_groups) {
  if (!p) return fail(PJ_ERR_ARG, "pj_plan_get_config: null plan");
  if (threads_per_block) *threads_per_block = p->tpb;
  if (blocks_per_sm) *blocks_per_sm = p->bps;
  if (use_shared) *use_shared = p->use_smem;
  if (n_groups) *n_groups = (int)p->groups.size();
  return PJ_OK;
}

extern "C" int pj_plan_run(pj_plan* p, void* stream) {
  if (!p) return fail(PJ_ERR_ARG, "pj_plan_run: null plan");
  return dispatch(p->op, p->mode, p->fmt, RunGroups{p, (cudaStream_t)stream});
}

extern "C" int pj_plan_capture(pj_plan* p, void* stream) {
  if (!p) return fail(PJ_ERR_ARG, "pj_plan_capture: null plan");
  if (!stream) return fail(PJ_ERR_ARG, "pj_plan_capture: needs a non-default stream");
  cudaStream_t st = (cudaStream_t)stream;
  drop_graph(p);
  cudaError_t e = cudaStreamBeginCapture(st, cudaStreamCaptureModeThreadLocal);
  if (e != cudaSuccess) return check_cuda(e, "cudaStreamBeginCapture");
  const int rc = dispatch(p->op, p->mode, p->fmt, RunGroups{p, st});
  cudaGraph_t g = nullptr;
  e = cudaStreamEndCapture(st, &g);
  if (rc) {
    if (g) cudaGraphDestroy(g);
    return rc;
  }
  if (e != cudaSuccess) return check_cuda(e, "cudaStreamEndCapture");
  p->graph = g;
  e = cudaGraphInstantiate(&p->exec, g, 0);
  if (e != cudaSuccess) {
    drop_graph(p);
    return check_cuda(e, "cudaGraphInstantiate");
  }
  return PJ_OK;
}

extern "C" int pj_plan_launch(pj_plan* p, void* stream) {
  if (!p) return fail(PJ_ERR_ARG, "pj_plan_launch: null plan");
  if (!p->exec) return fail(PJ_ERR_ARG, "pj_plan_launch: no captured graph (call pj_plan_capture)");
  return check_cuda(cudaGraphLaunch(p->exec, (cudaStream_t)stream), "cudaGraphLaunch");
}

extern "C" int pj_plan_autotune(pj_plan* p, void* stream, const char* cache_path, int reps) {
  if (!p) return fail(PJ_ERR_ARG, "pj_plan_autotune: null plan");
  cudaStream_t st = (cudaStream_t)stream;
  const std::string key = plan_key(p);
  int t0, b0, s0;
  if (cache_lookup(cache_path, key, &t0, &b0, &s0)) return plan_configure(p, t0, b0, s0);
  if (reps < 1) reps = 1;
  const size_t per_thread = (size_t)plan_arrays(p) * p->mech->ns * sizeof(double);
  struct Cand { int tpb, bps, sm; };
  std::vector<Cand> cands;
  for (int tpb : {32, 64, 128})
    for (int bps : {1, 2, 4, 8})
      for (int sm : {1, 0}) {
        if (sm && per_thread * tpb * bps > 225 * 1024) continue;
        if (!sm && per_thread * (size_t)tpb * bps * sm_count() > (size_t(8) << 30)) continue;  // workspace <= 8 GiB
        cands.push_back({tpb, bps, sm});
      }
  if (p->op == 1)  // the cooperative shapes (those that do not fit are skipped)
    for (int sm : {1, 0}) {
      cands.push_back({512, 1, sm});
      cands.push_back({256, 2, sm});
    }
  if (cands.empty()) cands.push_back({128, 1, 0});
  cudaEvent_t a, b;
  cudaEventCreate(&a);
  cudaEventCreate(&b);
  double best = 1e300;
  Cand bestc = cands[0];
  int rc = PJ_OK;
  for (const Cand& c : cands) {
    if ((rc = plan_configure(p, c.tpb, c.bps, c.sm))) {
      if (rc == PJ_ERR_UNSUPPORTED) continue;
      break;
    }
    if ((rc = pj_plan_run(p, st))) break;  // warm-up
    cudaEventRecord(a, st);
    for (int r = 0; r < reps && !rc; r++) rc = pj_plan_run(p, st);
    cudaEventRecord(b, st);
    if (rc) break;
    cudaError_t e = cudaEventSynchronize(b);
    if (e != cudaSuccess) {
      rc = check_cuda(e, "pj_plan_autotune: timing");
      break;
    }
    float ms = 0;
    cudaEventElapsedTime(&ms, a, b);
    if (ms / reps < best) {
      best = ms / reps;
      bestc = c;
    }
  }
  cudaEventDestroy(a);
  cudaEventDestroy(b);
  if (rc && rc != PJ_ERR_UNSUPPORTED) return rc;
  rc = plan_configure(p, bestc.tpb, bestc.bps, bestc.sm);
  if (!rc) cache_store(cache_path, key, bestc.tpb, bestc.bps, bestc.sm, best);
  return rc;
}
