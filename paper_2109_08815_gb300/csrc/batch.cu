// Batched execution of many inference problems: one persistent rollout
// launch per chain length over all problems' (particle, window) units, then
// each problem's window reduction and SVGD update on parallel graph
// branches; the whole iteration is captured once in a CUDA graph and
// replayed.  An autotuner picks, per chain length, the adjoint checkpoint
// stride, the math variant and the persistent grid size by timing the
// batched rollout itself.
#include <cuda_runtime.h>
#include <stdio.h>
#include <string.h>

#include <algorithm>
#include <vector>

#include "pds_internal.cuh"

namespace pds {

cudaError_t launch_batch_rollout(int NL, const BatchJob* jobs, const WorkItem* items, int n_items,
                                 unsigned int* counter, int grad, int fast, int blocks, int ring, int upt,
                                 cudaStream_t st) {
  switch (NL) {
    case 1: return launch_batch_rollout_nl<1>(jobs, items, n_items, counter, grad, fast, blocks, ring, upt, st);
    case 2: return launch_batch_rollout_nl<2>(jobs, items, n_items, counter, grad, fast, blocks, ring, upt, st);
    case 3: return launch_batch_rollout_nl<3>(jobs, items, n_items, counter, grad, fast, blocks, ring, upt, st);
    case 4: return launch_batch_rollout_nl<4>(jobs, items, n_items, counter, grad, fast, blocks, ring, upt, st);
    case 5: return launch_batch_rollout_nl<5>(jobs, items, n_items, counter, grad, fast, blocks, ring, upt, st);
    case 6: return launch_batch_rollout_nl<6>(jobs, items, n_items, counter, grad, fast, blocks, ring, upt, st);
    case 7: return launch_batch_rollout_nl<7>(jobs, items, n_items, counter, grad, fast, blocks, ring, upt, st);
    case 8: return launch_batch_rollout_nl<8>(jobs, items, n_items, counter, grad, fast, blocks, ring, upt, st);
    default: return cudaErrorInvalidValue;
  }
}

static int blocks_per_sm(int NL, int fast, int upt) {
  switch (NL) {
    case 1: return batch_rollout_blocks_per_sm_nl<1>(fast, upt);
    case 2: return batch_rollout_blocks_per_sm_nl<2>(fast, upt);
    case 3: return batch_rollout_blocks_per_sm_nl<3>(fast, upt);
    case 4: return batch_rollout_blocks_per_sm_nl<4>(fast, upt);
    case 5: return batch_rollout_blocks_per_sm_nl<5>(fast, upt);
    case 6: return batch_rollout_blocks_per_sm_nl<6>(fast, upt);
    case 7: return batch_rollout_blocks_per_sm_nl<7>(fast, upt);
    case 8: return batch_rollout_blocks_per_sm_nl<8>(fast, upt);
    default: return 1;
  }
}

// All problems of one chain length.
struct Group {
  int NL = 0;
  std::vector<int> jobs;          // indices into the batch
  int K = 10, fast = 0, blocks = 0;
  int upt = 0;                    // rollout units per thread: 1, 2, or 0 = by chain length (2, 4, 5 links: two)
  bool pair = false;              // the built tables are for two units per thread
  BatchJob* d_jobs = nullptr;
  WorkItem* d_items = nullptr;
  int n_items = 0;
  unsigned int* d_counter = nullptr;
};

}  // namespace pds

using namespace pds;

struct pds_batch {
  std::vector<pds_problem*> probs;
  std::vector<pds_svgd*> svgds;
  std::vector<float*> X;
  std::vector<float*> logp;       // caller's per-problem log p outputs (may be NULL)
  std::vector<Group> groups;
  cudaStream_t stream = nullptr;  // the batch's own stream (captured into the graph)
  cudaStream_t user = nullptr;    // the caller's stream; joined through events
  cudaEvent_t ev_in = nullptr, ev_out = nullptr;
  std::vector<cudaStream_t> side;
  std::vector<cudaEvent_t> ev;    // [0] fork, [1..] joins
  std::vector<cudaStream_t> gstream;  // one branch per chain-length group's rollout
  std::vector<cudaEvent_t> gdone;     // that rollout finished
  std::vector<int> group_of;          // problem -> its group (-1: rolled out on its own branch)
  cudaGraphExec_t exec = nullptr;
  cudaGraph_t graph = nullptr;
  bool dirty = true;              // tables or settings changed since the graph was captured
  bool eager_done = false;        // the first iteration after a rebuild runs without a graph
  int sm_count = 0;
  int launches_per_iter = 0;
};

// Parallel graph branches for the problems' reductions and SVGD steps: one
// per problem up to this many.  A small problem's step is a chain of short
// launches that leave most of the GPU idle, so more branches overlap more of
// them (64 uneven problems: 4.56 ms per iteration with 8 branches, 3.59 ms
// with 32).
static constexpr int kMaxSideStreams = 64;

static void free_group(Group& g) {
  cudaFree(g.d_jobs);
  cudaFree(g.d_items);
  cudaFree(g.d_counter);
  g.d_jobs = nullptr;
  g.d_items = nullptr;
  g.d_counter = nullptr;
}

static void drop_graph(pds_batch* b) {
  if (b->exec) cudaGraphExecDestroy(b->exec);
  if (b->graph) cudaGraphDestroy(b->graph);
  b->exec = nullptr;
  b->graph = nullptr;
}

// (Re)build a group's device job table and cost-ordered work list.
static int build_group(pds_batch* b, Group& g) {
  free_group(g);
  // two units per thread: asked for (or by default for the chain lengths
  // where the single-problem kernel measured faster) and possible for every
  // problem of the group (K = 1, every state component observed, even N)
  bool pair = g.upt == 2 || (g.upt == 0 && (g.NL == 2 || g.NL == 4 || g.NL == 5));
  pair = pair && g.K == 1;
  for (size_t a = 0; a < g.jobs.size() && pair; ++a) {
    const pds_problem* p = b->probs[g.jobs[a]];
    const unsigned int all = (1u << (2 * g.NL)) - 1u;
    pair = (p->c.obs_mask & all) == all && p->c.obs_b != nullptr && !p->c.csvgd &&
           b->svgds[g.jobs[a]]->sp.N % 2 == 0;
  }
  const int span = pair ? 256 : 128;  // units per work item
  std::vector<BatchJob> jobs;
  struct Item { WorkItem w; int cost; };
  std::vector<Item> items;
  for (size_t a = 0; a < g.jobs.size(); ++a) {
    pds_problem* p = b->probs[g.jobs[a]];
    p->c.K = g.K;
    p->c.fast_math = g.fast;
    // checkpoint slots depend on K
    int hmax = 0;
    for (int w = 0; w < p->c.W; ++w) {
      const int h = (int)(((long long)(w + 1) * p->c.T) / p->c.W - ((long long)w * p->c.T) / p->c.W);
      hmax = std::max(hmax, h);
    }
    p->c.max_seg = (hmax + p->c.K - 1) / p->c.K;
    const int N = b->svgds[g.jobs[a]]->sp.N;
    int rc = ensure_workspace(p, N);
    if (rc != PDS_OK) return rc;
    rc = ensure_iter_buffers(p, N);
    if (rc != PDS_OK) return rc;
    BatchJob bj;
    memset(&bj, 0, sizeof(bj));
    bj.c = p->c;
    bj.X = b->X[g.jobs[a]];
    bj.N = N;
    bj.parts = p->parts;
    bj.status = nullptr;
    jobs.push_back(bj);
    const long long U = (long long)N * p->c.W;
    for (long long u0 = 0; u0 < U; u0 += span) {
      const long long u1 = std::min(U, u0 + span) - 1;
      int cost = 0;
      for (long long w = u0 / N; w <= u1 / N; ++w) {
        const int h = (int)(((w + 1) * p->c.T) / p->c.W - (w * p->c.T) / p->c.W);
        cost = std::max(cost, h);
      }
      items.push_back({{(int)a, (int)u0}, cost});
    }
  }
  std::stable_sort(items.begin(), items.end(), [](const Item& x, const Item& y) { return x.cost > y.cost; });
  std::vector<WorkItem> w(items.size());
  for (size_t k = 0; k < items.size(); ++k) w[k] = items[k].w;
  g.n_items = (int)w.size();
  cudaError_t e;
  if ((e = cudaMalloc(&g.d_jobs, jobs.size() * sizeof(BatchJob))) != cudaSuccess ||
      (e = cudaMalloc(&g.d_items, std::max<size_t>(1, w.size()) * sizeof(WorkItem))) != cudaSuccess ||
      (e = cudaMalloc(&g.d_counter, sizeof(unsigned int))) != cudaSuccess) {
    free_group(g);
    return set_error(PDS_ERR_OOM, "batch table allocation failed");
  }
  if ((e = cudaMemcpy(g.d_jobs, jobs.data(), jobs.size() * sizeof(BatchJob), cudaMemcpyHostToDevice)) !=
          cudaSuccess ||
      (w.size() && (e = cudaMemcpy(g.d_items, w.data(), w.size() * sizeof(WorkItem), cudaMemcpyHostToDevice)) !=
                       cudaSuccess))
    return set_error(PDS_ERR_CUDA, "batch table upload failed");
  g.pair = pair;
  if (g.blocks <= 0) g.blocks = b->sm_count * std::max(1, blocks_per_sm(g.NL, g.fast, pair ? 2 : 1));
  return PDS_OK;
}

static cudaError_t launch_group_rollout(Group& g, cudaStream_t st) {
  cudaError_t e = cudaMemsetAsync(g.d_counter, 0, sizeof(unsigned int), st);
  if (e != cudaSuccess) return e;
  return launch_batch_rollout(g.NL, g.d_jobs, g.d_items, g.n_items, g.d_counter, 1, g.fast, g.blocks, g.K == 1 ? 1 : 0,
                              g.pair ? 2 : 1, st);
}

// One iteration of every problem: the chain-length groups' rollouts on
// branches of their own (persistent kernels that take work from a counter,
// so concurrent groups fill one another's tails), each problem's reduction
// and SVGD step on a side branch that waits only for its own group.
static cudaError_t enqueue_iteration(pds_batch* b, int* launches) {
  int n = 0;
  cudaError_t e;
  if ((e = cudaEventRecord(b->ev[0], b->stream)) != cudaSuccess) return e;
  for (size_t gi = 0; gi < b->groups.size(); ++gi) {
    cudaStream_t gs = b->gstream[gi];
    if ((e = cudaStreamWaitEvent(gs, b->ev[0], 0)) != cudaSuccess) return e;
    if ((e = launch_group_rollout(b->groups[gi], gs)) != cudaSuccess) return e;
    if ((e = cudaEventRecord(b->gdone[gi], gs)) != cudaSuccess) return e;
    ++n;
  }
  const int n_side = (int)b->side.size();
  for (int s = 0; s < n_side; ++s)
    if ((e = cudaStreamWaitEvent(b->side[s], b->ev[0], 0)) != cudaSuccess) return e;
  for (size_t j = 0; j < b->probs.size(); ++j) {
    pds_problem* p = b->probs[j];
    pds_svgd* s = b->svgds[j];
    cudaStream_t st = b->side[j % n_side];
    SvgdWork w = s->w;
    if (s->full_passes) {
      w.cand_cap = 0;
      w.small_median = 0;
    }
    if (s->phi_cuda_cores) w.tc = nullptr;
    if (s->median_cuda_cores) w.mimg = nullptr;
    // a step that takes the sampled median bracket starts its median phase
    // (coordinates only) before the rollout of its chain length is done
    const bool split = svgd_step_splits(s->sp, w) && !s->grad_dead_seen;
    int k = 0;
    if (split && (e = launch_svgd_step(s->sp, w, b->X[j], p->d_grad, nullptr, nullptr, st, &k, kSvgdTheta)) != cudaSuccess)
      return e;
    if (b->group_of[j] >= 0 && (e = cudaStreamWaitEvent(st, b->gdone[b->group_of[j]], 0)) != cudaSuccess) return e;
    const int N = s->sp.N;
    float* lp = b->logp[j] ? b->logp[j] : p->d_logp;
    if (p->kind == PDS_SYSTEM_ARM_BOX) {
      // not part of the chain-length groups: its own rollout on the branch
      if ((e = launch_armbox_rollout(p->c, p->ab, b->X[j], N, p->parts, 1, nullptr, st)) != cudaSuccess) return e;
      ++n;
    } else if (p->kind == PDS_SYSTEM_RIGID_DOUBLE_PENDULUM) {
      if ((e = launch_rigid2_rollout(p->c, p->r2, b->X[j], N, p->parts, 1, nullptr, st)) != cudaSuccess) return e;
      ++n;
    }
    if ((e = launch_window_reduce(p->c, b->X[j], N, p->parts, lp, p->d_grad, nullptr, st)) != cudaSuccess)
      return e;
    if ((e = launch_svgd_step(s->sp, w, b->X[j], p->d_grad, nullptr, nullptr, st, &k,
                              split ? kSvgdGrad : kSvgdAll)) != cudaSuccess)
      return e;
    n += 1 + k;
  }
  for (int s = 0; s < n_side; ++s) {
    if ((e = cudaEventRecord(b->ev[1 + s], b->side[s])) != cudaSuccess) return e;
    if ((e = cudaStreamWaitEvent(b->stream, b->ev[1 + s], 0)) != cudaSuccess) return e;
  }
  for (size_t gi = 0; gi < b->groups.size(); ++gi)
    if ((e = cudaStreamWaitEvent(b->stream, b->gdone[gi], 0)) != cudaSuccess) return e;
  if (launches) *launches = n;
  return cudaSuccess;
}

// Rebuild the job tables if anything changed (drops the captured graph).
static int rebuild(pds_batch* b) {
  if (!b->dirty) return PDS_OK;
  drop_graph(b);
  for (Group& g : b->groups) {
    int rc = build_group(b, g);
    if (rc != PDS_OK) return rc;
  }
  for (size_t j = 0; j < b->probs.size(); ++j) {
    if (b->probs[j]->kind == PDS_SYSTEM_PLANAR_CHAIN) continue;
    int rc = ensure_workspace(b->probs[j], b->svgds[j]->sp.N);
    if (rc == PDS_OK) rc = ensure_iter_buffers(b->probs[j], b->svgds[j]->sp.N);
    if (rc != PDS_OK) return rc;
  }
  b->dirty = false;
  b->eager_done = false;
  return PDS_OK;
}

static int capture(pds_batch* b) {
  cudaError_t e = cudaStreamBeginCapture(b->stream, cudaStreamCaptureModeThreadLocal);
  if (e != cudaSuccess) return set_error(PDS_ERR_CUDA, "batch: begin capture failed");
  int n = 0;
  cudaError_t el = enqueue_iteration(b, &n);
  e = cudaStreamEndCapture(b->stream, &b->graph);
  if (el != cudaSuccess || e != cudaSuccess) {
    drop_graph(b);
    return set_error(PDS_ERR_CUDA, "batch: capture of the iteration failed");
  }
  e = cudaGraphInstantiate(&b->exec, b->graph, 0);
  if (e != cudaSuccess) {
    drop_graph(b);
    return set_error(PDS_ERR_CUDA, "batch: graph instantiation failed");
  }
  b->launches_per_iter = n;
  return PDS_OK;
}

extern "C" {

int pds_batch_create(int n_jobs, pds_problem_t const* problems, pds_svgd_t const* svgds, float* const* particles,
                     float* const* logp, void* cuda_stream, pds_batch_t* out) {
  if (!out) return set_error(PDS_ERR_ARG, "out is NULL");
  *out = nullptr;
  if (n_jobs < 1 || !problems || !svgds || !particles) return set_error(PDS_ERR_ARG, "bad batch arguments");
  pds_batch* b = new pds_batch();
  b->user = (cudaStream_t)cuda_stream;
  // a stream of its own: the caller's may be the legacy default stream,
  // which cannot be captured
  if (cudaStreamCreateWithFlags(&b->stream, cudaStreamNonBlocking) != cudaSuccess ||
      cudaEventCreateWithFlags(&b->ev_in, cudaEventDisableTiming) != cudaSuccess ||
      cudaEventCreateWithFlags(&b->ev_out, cudaEventDisableTiming) != cudaSuccess) {
    delete b;
    return set_error(PDS_ERR_CUDA, "batch: stream creation failed");
  }
  int dev = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&b->sm_count, cudaDevAttrMultiProcessorCount, dev);
  for (int j = 0; j < n_jobs; ++j) {
    pds_problem* p = problems[j];
    pds_svgd* s = svgds[j];
    if (!p || !s || !particles[j]) {
      delete b;
      return set_error(PDS_ERR_ARG, "NULL problem, SVGD state or particle buffer in the batch");
    }
    if (s->sp.M != p->c.M || s->sp.P != p->c.P) {
      delete b;
      return set_error(PDS_ERR_ARG, "SVGD state does not match its problem");
    }
    if (p->c.csvgd || s->sp.csvgd || p->c.R > 1) {
      delete b;
      return set_error(PDS_ERR_UNSUPPORTED, "batched execution runs the unconstrained one-trajectory method only");
    }
    if (p->kind != PDS_SYSTEM_PLANAR_CHAIN && p->kind != PDS_SYSTEM_ARM_BOX &&
        p->kind != PDS_SYSTEM_RIGID_DOUBLE_PENDULUM) {
      delete b;
      return set_error(PDS_ERR_UNSUPPORTED, "unknown system kind in the batch");
    }
    b->probs.push_back(p);
    b->svgds.push_back(s);
    b->X.push_back(particles[j]);
    b->logp.push_back(logp ? logp[j] : nullptr);
  }
  for (int nl = 1; nl <= PDS_MAX_LINKS; ++nl) {
    Group g;
    g.NL = nl;
    for (int j = 0; j < n_jobs; ++j)
      if (b->probs[j]->kind == PDS_SYSTEM_PLANAR_CHAIN && b->probs[j]->c.n == nl) g.jobs.push_back(j);
    if (!g.jobs.empty()) {
      g.K = b->probs[g.jobs[0]]->c.K;
      g.fast = b->probs[g.jobs[0]]->c.fast_math;
      g.upt = b->probs[g.jobs[0]]->c.units_per_thread;
      b->groups.push_back(g);
    }
  }
  b->group_of.assign(n_jobs, -1);
  for (size_t gi = 0; gi < b->groups.size(); ++gi)
    for (int j : b->groups[gi].jobs) b->group_of[j] = (int)gi;
  for (size_t gi = 0; gi < b->groups.size(); ++gi) {
    cudaStream_t gs = nullptr;
    cudaEvent_t ge = nullptr;
    if (cudaStreamCreateWithFlags(&gs, cudaStreamNonBlocking) != cudaSuccess) {
      pds_batch_destroy(b);
      return set_error(PDS_ERR_CUDA, "batch: stream creation failed");
    }
    b->gstream.push_back(gs);
    if (cudaEventCreateWithFlags(&ge, cudaEventDisableTiming) != cudaSuccess) {
      pds_batch_destroy(b);
      return set_error(PDS_ERR_CUDA, "batch: event creation failed");
    }
    b->gdone.push_back(ge);
  }
  const int n_side = n_jobs < kMaxSideStreams ? n_jobs : kMaxSideStreams;
  b->side.resize(n_side);
  b->ev.resize(1 + n_side);
  for (int s = 0; s < n_side; ++s)
    if (cudaStreamCreateWithFlags(&b->side[s], cudaStreamNonBlocking) != cudaSuccess) {
      b->side.resize(s);
      b->ev.clear();
      pds_batch_destroy(b);
      return set_error(PDS_ERR_CUDA, "batch: stream creation failed");
    }
  for (auto& e : b->ev) cudaEventCreateWithFlags(&e, cudaEventDisableTiming);
  *out = b;
  return PDS_OK;
}

int pds_batch_destroy(pds_batch_t b) {
  if (!b) return PDS_OK;
  cudaStreamSynchronize(b->stream);
  drop_graph(b);
  for (Group& g : b->groups) free_group(g);
  for (auto s : b->side) cudaStreamDestroy(s);
  for (auto e : b->ev) cudaEventDestroy(e);
  for (auto s : b->gstream) cudaStreamDestroy(s);
  for (auto e : b->gdone) cudaEventDestroy(e);
  cudaEventDestroy(b->ev_in);
  cudaEventDestroy(b->ev_out);
  cudaStreamDestroy(b->stream);
  delete b;
  return PDS_OK;
}

int pds_batch_autotune(pds_batch_t b, int allow_fast_math, int* choices) {
  if (!b) return set_error(PDS_ERR_ARG, "NULL batch");
  cudaStreamSynchronize(b->user);
  cudaEvent_t t0, t1;
  cudaEventCreate(&t0);
  cudaEventCreate(&t1);
  const int Ks[] = {1, 5, 10, 25, 50};
  int gi = 0;
  for (Group& g : b->groups) {
    int best_K = g.K, best_fast = g.fast, best_blocks = 0, best_upt = 1;
    float best = 1e30f;
    for (int fast = 0; fast <= (allow_fast_math ? 1 : 0); ++fast) {
      for (int K : Ks) {
        // K = 1 also with two units per thread (taken only where every
        // problem of the group allows it)
        for (int upt = 1; upt <= (K == 1 ? 2 : 1); ++upt) {
          g.K = K;
          g.fast = fast;
          g.upt = upt;
          g.blocks = 0;
          int rc = build_group(b, g);
          if (rc != PDS_OK) return rc;
          if (upt == 2 && !g.pair) continue;
          const int occ = std::max(1, blocks_per_sm(g.NL, fast, upt));
          for (int per_sm = occ; per_sm >= std::max(1, occ - 1); --per_sm) {
            g.blocks = b->sm_count * per_sm;
            float ms = 0.f, tot = 0.f;
            for (int r = 0; r < 4; ++r) {
              cudaEventRecord(t0, b->stream);
              if (launch_group_rollout(g, b->stream) != cudaSuccess)
                return set_error(PDS_ERR_CUDA, "autotune launch failed");
              cudaEventRecord(t1, b->stream);
              cudaEventSynchronize(t1);
              cudaEventElapsedTime(&ms, t0, t1);
              if (r > 0) tot += ms;  // the first run warms up
            }
            if (tot < best) {
              best = tot;
              best_K = K;
              best_fast = fast;
              best_blocks = g.blocks;
              best_upt = upt;
            }
          }
        }
      }
    }
    g.K = best_K;
    g.fast = best_fast;
    g.upt = best_upt;
    g.blocks = best_blocks;
    if (choices) {
      choices[5 * gi + 0] = g.NL;
      choices[5 * gi + 1] = g.K;
      choices[5 * gi + 2] = g.fast;
      choices[5 * gi + 3] = g.blocks;
      choices[5 * gi + 4] = g.upt;
    }
    ++gi;
  }
  cudaEventDestroy(t0);
  cudaEventDestroy(t1);
  b->dirty = true;
  return PDS_OK;
}

int pds_batch_iterate(pds_batch_t b, int iters) {
  if (!b) return set_error(PDS_ERR_ARG, "NULL batch");
  if (iters < 0) return set_error(PDS_ERR_ARG, "iters < 0");
  int rc = rebuild(b);
  if (rc != PDS_OK) return rc;
  cudaError_t e = svgd_setup_device();
  if (e != cudaSuccess) return set_error(PDS_ERR_CUDA, "batch: device set-up failed");
  // order after the caller's earlier work, and the caller's later work after ours
  if ((e = cudaEventRecord(b->ev_in, b->user)) != cudaSuccess ||
      (e = cudaStreamWaitEvent(b->stream, b->ev_in, 0)) != cudaSuccess)
    return set_error(PDS_ERR_CUDA, "batch: stream join failed");
  int launches = 0;
  for (int it = 0; it < iters; ++it) {
    if (!b->exec && !b->eager_done) {
      // first iteration after a (re)build: plain launches, no capture cost
      int n = 0;
      if ((e = enqueue_iteration(b, &n)) != cudaSuccess) return set_error(PDS_ERR_CUDA, "batch: launch failed");
      b->launches_per_iter = n;
      b->eager_done = true;
      launches += n;
      continue;
    }
    if (!b->exec) {
      rc = capture(b);
      if (rc != PDS_OK) return rc;
    }
    if ((e = cudaGraphLaunch(b->exec, b->stream)) != cudaSuccess)
      return set_error(PDS_ERR_CUDA, "batch: graph launch failed");
    launches += b->launches_per_iter;
  }
  if ((e = cudaEventRecord(b->ev_out, b->stream)) != cudaSuccess ||
      (e = cudaStreamWaitEvent(b->user, b->ev_out, 0)) != cudaSuccess)
    return set_error(PDS_ERR_CUDA, "batch: stream join failed");
  set_launch_count(launches);
  return PDS_OK;
}

int pds_batch_info(pds_batch_t b, int* n_groups, int* launches_per_iter) {
  if (!b) return set_error(PDS_ERR_ARG, "NULL batch");
  if (n_groups) *n_groups = (int)b->groups.size();
  if (launches_per_iter) *launches_per_iter = b->launches_per_iter;
  return PDS_OK;
}

}  // extern "C"
