// bbc_api.cpp -- C ABI of libbbc (declared in include/bbc.h).
//
// A context owns the host plan (planner.cpp) and a view of the caller's
// device workspace: the plan tables, per-slot propagator copies and the
// block fields of every slot.  Every device operation is issued on the
// context stream; nothing here allocates device memory.
#include "../../include/bbc.h"

#include <cmath>
#include <cstring>
#include <map>
#include <mutex>
#include <new>
#include <string>
#include <vector>

#include <cuda_runtime.h>
#include <nvtx3/nvToolsExt.h>

#include "ctx_internal.hpp"
#include "kernels.cuh"
#include "planner.hpp"

namespace {

std::string g_create_error;

size_t align256(size_t x) { return (x + 255) & ~size_t(255); }
// FP64 storage (plain FP64, and FP64 with double-float products) or FP32
bool fp64_storage(int prec) { return prec == BBC_FP64 || prec == BBC_DF64; }
size_t cplx_bytes(int prec) { return fp64_storage(prec) ? 16 : 8; }
bool fused_path(int prec) { return !fp64_storage(prec); }  // FP32 or bfloat16 products (if they fit one CTA)
// The fused FP32 path's forward FFT runs as one queue-driven persistent launch for L <= 32.
bool queue_fft(const bbc_ctx* c) { return c->fused && bbc::fft_queue_supported(c->lat.L); }
int real_kind(int prec) { return prec == BBC_DF64 ? bbc::RK_DF : (prec == BBC_FP64 ? bbc::RK_F64 : bbc::RK_F32); }

constexpr int kMaxFusedWarps = 16;
// tensor-core contexts: precisions whose trace-form block pairs run on the tensor cores
bool tensor_path(int prec) { return prec == BBC_MIXED_FP32 || prec == BBC_MIXED_TF32; }
// Warp task lists of the block-pair products per 32 q (autotuned).
const int kPairGroupsCand[] = {48, 96, 192, 384};
constexpr int kMaxPairGroups = 384;

struct Layout {
  size_t ell_chunk, ell, zneed, tasks, group_ptr, group_task, cptr, citem, ccoef, ccoef_df;
  size_t batches, wptr, wunits, qlist, row_slot, orb_ptr, orb_site;
  size_t tc_base, tc_units, row_map, tc_cptr, tc_terms, tc_coefs, dtuples, dchunk, dell, tables_end;
  size_t stage, prop, amax, kexp, blk, blk16, blkf, blks, P, G, ct, scale, flag, qerr, fftq, total;
};

Layout layout(const bbc_ctx* c, int slots) {
  const bbc::Plan& p = c->plan;
  Layout L{};
  size_t o = 0;
  L.ell_chunk = o; o = align256(o + sizeof(int2) * p.ell_chunk.size());
  L.ell = o; o = align256(o + sizeof(uint32_t) * p.ell.size());
  L.zneed = o; o = align256(o + sizeof(uint32_t) * p.zneed.size());
  L.tasks = o; o = align256(o + sizeof(bbc::DevTask) * p.tasks.size());
  L.group_ptr = o; o = align256(o + sizeof(int) * (kMaxPairGroups + 1));
  L.group_task = o; o = align256(o + sizeof(int) * c->group_task.size());
  L.cptr = o; o = align256(o + sizeof(int) * p.tcontrib_ptr.size());
  L.citem = o; o = align256(o + sizeof(int) * p.tcontrib_item.size());
  L.ccoef = o; o = align256(o + sizeof(double) * p.tcontrib_coef.size());
  L.ccoef_df = o; o = align256(o + (c->prec == BBC_DF64 ? sizeof(float2) * p.tcontrib_coef.size() : 0));
  L.batches = o; o = align256(o + sizeof(bbc::WarpBatch) * c->batches.size());
  L.wptr = o; o = align256(o + sizeof(int) * (kMaxFusedWarps + 1));
  L.wunits = o; o = align256(o + sizeof(int4) * c->max_units);
  L.qlist = o; o = align256(o + sizeof(int) * c->qlist.size());
  L.row_slot = o; o = align256(o + sizeof(int) * c->row_slot.size());
  L.orb_ptr = o; o = align256(o + sizeof(int) * c->orb_ptr.size());
  L.orb_site = o; o = align256(o + sizeof(int) * c->orb_site.size());
  L.tc_base = o; o = align256(o + sizeof(int) * c->tcs.base.size());
  L.tc_units = o; o = align256(o + sizeof(int) * c->tcs.units.size());
  L.row_map = o; o = align256(o + sizeof(uint32_t) * c->tcs.row_src.size());
  L.tc_cptr = o; o = align256(o + sizeof(int) * c->tcs.out_ptr.size());
  L.tc_terms = o; o = align256(o + sizeof(uint2) * c->tcs.coef.size());
  L.tc_coefs = o; o = align256(o + sizeof(float2) * c->tcs.coef_values.size());
  L.dtuples = o; o = align256(o + sizeof(uint32_t) * c->db.tuples.size());
  L.dchunk = o; o = align256(o + sizeof(int2) * c->db.ell_chunk.size());
  L.dell = o; o = align256(o + sizeof(uint32_t) * c->db.ell.size());
  L.tables_end = o;
  const size_t V = c->V;
  L.stage = o; o = align256(o + (size_t)slots * 2 * V * 144 * 16);
  L.prop = o; o = align256(o + (size_t)slots * 2 * V * 144 * cplx_bytes(c->prec));
  L.amax = o; o = align256(o + (size_t)slots * 2 * sizeof(unsigned long long));
  L.kexp = o; o = align256(o + (size_t)slots * 2 * sizeof(int));
  L.blk = o; o = align256(o + (size_t)slots * V * p.n_out * cplx_bytes(c->prec));
  L.blk16 = o; o = align256(o + (c->prec == BBC_MIXED_BF16 ? (size_t)slots * V * p.n_out * 4 : 0));
  const bool split = !c->fused;  // the fused path keeps q-major blocks and no product buffer
  L.blkf = o; o = align256(o + (split ? (size_t)slots * V * p.n_out * cplx_bytes(c->prec) : 0));
  // FP64: re + im of every Fourier-space block value (the FP64 products' sums)
  L.blks = o; o = align256(o + (c->prec == BBC_FP64 ? (size_t)slots * V * p.n_out * sizeof(double) : 0));
  L.P = o; o = align256(o + (split ? (size_t)p.tasks.size() * 16 * V * cplx_bytes(c->prec) : 0));
  // tensor-core products of one slice: G(q) per pair {q, -q}, complex64
  L.G = o; o = align256(o + (c->tc ? c->qlist.size() * (size_t)c->tcs.nbp * c->tcs.nbp * 8 : 0));
  L.ct = o; o = align256(o + (size_t)p.channels.size() * 16 * V * 16);
  L.scale = o; o = align256(o + sizeof(double) * bbc::kMaxChannels);
  L.flag = o; o = align256(o + sizeof(int));
  // queue-driven forward FFT: its sticky timeout word, ticket counter and per-tile counters
  L.qerr = o; o = align256(o + sizeof(int));
  L.fftq = o; o = align256(o + (queue_fft(c) ? sizeof(int) * bbc::fft_queue_ints(c->lat.L, slots, p.n_out) : 0));
  L.total = o;
  return L;
}

bbc_status fail(const bbc_ctx* c, bbc_status s, const std::string& m) {
  if (c) c->err = m;
  else g_create_error = m;
  return s;
}

bbc_status cuda_fail(bbc_ctx* c, cudaError_t e, const char* where) {
  return fail(c, BBC_ECUDA, std::string(where) + ": " + cudaGetErrorString(e));
}

// Time distance of slice t from the source: forward (t - t0) mod T for the
// upper components, backward (t0 - t) mod T for the lower ones (Sec. 5).
int time_distance(const bbc_ctx* c, int t) {
  const int T = c->lat.T, dt = c->plan.spin_offset ? c->lat.t0 - t : t - c->lat.t0;
  return ((dt % T) + T) % T;
}

bool supported_L(int L) { return L == 2 || L == 4 || L == 8 || L == 16 || L == 24 || L == 32 || L == 48; }

cudaEvent_t take_event(bbc_ctx* c) {
  if (!c->pool.empty()) {
    cudaEvent_t e = c->pool.back();
    c->pool.pop_back();
    return e;
  }
  cudaEvent_t e = nullptr;
  if (cudaEventCreate(&e) != cudaSuccess) return nullptr;
  return e;
}

// NVTX range names of the stages (host-side launch ranges, visible to
// profilers that attach an NVTX tool; no-ops otherwise).
const char* const kStageRange[BBC_N_STAGES] = {"bbc ingest",  "bbc build",     "bbc fft_fwd", "bbc contract",
                                               "bbc fft_inv", "bbc normalise", "bbc wick",    "bbc project"};

// Brackets one stage launch with an NVTX range, and with events when timing
// is enabled.
struct StageScope {
  bbc_ctx* c;
  int stage;
  cudaEvent_t a = nullptr, b = nullptr;
  StageScope(bbc_ctx* ctx, int s) : c(ctx), stage(s) {
    nvtxRangePushA(kStageRange[s]);
    if (!c->timing) return;
    a = take_event(c);
    b = take_event(c);
    if (a) cudaEventRecord(a, c->stream);
  }
  ~StageScope() {
    if (a && b) {
      cudaEventRecord(b, c->stream);
      c->pending[stage].push_back({a, b});
    }
    nvtxRangePop();
  }
};

// Warp batches and shared-memory bank layout of the fused contraction depend
// on the channel list only; computed once per list and process.
struct FusedSchedule {
  std::vector<bbc::Batch> batches;
  bbc::FusedLayout layout;
};
std::mutex g_sched_mutex;
std::map<std::vector<int>, FusedSchedule> g_sched;

// A plan is fixed by its channel list and spin components.
std::vector<int> plan_key(const bbc::Plan& plan) {
  std::vector<int> k = plan.channels;
  k.push_back(-1 - plan.spin_offset);
  return k;
}

// The plan the fused kernels run: the whole plan, or (tensor-core contexts)
// the tasks left to the CUDA cores on their compact rows.
const bbc::Plan& fused_plan(const bbc_ctx* c) { return c->tc ? c->tcs.rest : c->plan; }

// plan: the context's plan (the cache key); run: the plan the kernel runs
const FusedSchedule& fused_schedule(const bbc::Plan& plan, const bbc::Plan& run, bool tc) {
  std::lock_guard<std::mutex> lock(g_sched_mutex);
  std::vector<int> key = plan_key(plan);
  if (tc) key.push_back(-100);
  auto it = g_sched.find(key);
  if (it != g_sched.end()) return it->second;
  FusedSchedule f;
  bbc::make_batches(run, &f.batches);
  bbc::optimise_fused_layout(run, &f.batches, &f.layout);
  return g_sched.emplace(key, std::move(f)).first->second;
}

// Candidate launch configurations of the autotuner.
const int kBuildCand[][2] = {{1, 256}, {2, 256}, {2, 512}, {4, 512}, {1, 512}};  // (sites per CTA, threads)
const int kFusedWarpsCand[] = {8, 12, 16};
const int kRestWarpsCand[] = {4, 8};  // k_contract_rest (two CTAs per SM)
const int kFusedStepsCand[] = {1, 2};
const int kChunkCand[] = {0, 18, 36, 72, 144};  // 0: contiguous equal-cost pieces

// Tuned configurations per (L, precision, channel list), for later contexts.
std::mutex g_tune_mutex;
std::map<std::pair<std::pair<int, int>, std::vector<int>>, bbc_tuning> g_tuned;

bool tuning_valid(const bbc_ctx* c, const bbc_tuning& t) {
  if (!bbc::build_variant_supported(t.build_sites, t.build_threads) || c->V % t.build_sites != 0) return false;
  bool groups_ok = false;
  for (int g : kPairGroupsCand) groups_ok |= g == t.pair_groups;
  if (!groups_ok || (t.tc_kernel != 0 && t.tc_kernel != 1)) return false;
  if (c->dense) {
    if (!bbc::dense_build_supported(t.build_sites, t.build_threads) ||
        bbc::dense_build_smem(bbc::dev_groups(c->plan, &c->db), t.build_sites) > bbc::kMaxSmemPerBlock)
      return false;
  } else if (bbc::block_build_smem(c->plan.z_slots, t.build_sites, fp64_storage(c->prec),
                                   (int)c->plan.diquarks.size()) > bbc::kMaxSmemPerBlock) {
    return false;
  }
  if (c->fused) {
    if (c->tc ? !bbc::rest_variant_supported(t.fused_warps, t.fused_steps)
              : !bbc::fused_variant_supported(t.fused_warps, t.fused_steps))
      return false;
    bool chunk_ok = false;
    for (int k : kChunkCand) chunk_ok |= k == t.fused_chunk;
    if (!chunk_ok) return false;
  }
  return true;
}

// Task lists of the block-pair products for the context's pair_groups,
// uploaded when a workspace is attached (synchronous).
// (The host lists exist for fused contexts too: the static entry point runs
// the unfused products for them.)
bbc_status apply_pair_groups(bbc_ctx* c) {
  bbc::make_task_groups(c->plan, c->tune.pair_groups, &c->group_ptr, &c->group_task, c->prec == BBC_DF64);
  if ((int)c->group_ptr.size() > kMaxPairGroups + 1 || c->group_task.size() != c->plan.tasks.size())
    return fail(c, BBC_EINVAL, "internal: task groups exceed their workspace");
  if (!c->ws || c->fused) return BBC_OK;
  cudaError_t e = cudaMemcpyAsync(c->d_group_ptr, c->group_ptr.data(), sizeof(int) * c->group_ptr.size(),
                                  cudaMemcpyHostToDevice, c->stream);
  if (e == cudaSuccess && !c->group_task.empty())
    e = cudaMemcpyAsync(c->d_group_task, c->group_task.data(), sizeof(int) * c->group_task.size(),
                        cudaMemcpyHostToDevice, c->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
  if (e != cudaSuccess) return cuda_fail(c, e, "task group upload");
  return BBC_OK;
}

// Warp units of the context's fused configuration, uploaded when a
// workspace is attached (synchronous: the host vectors are temporaries).
bbc_status apply_fused_units(bbc_ctx* c) {
  if (!c->fused) return BBC_OK;
  const FusedSchedule& f = fused_schedule(c->plan, fused_plan(c), c->tc);
  bbc::make_units(fused_plan(c), f.batches, c->tune.fused_warps, c->tune.fused_chunk, &c->wptr, &c->wunits);
  if (c->wunits.size() > c->max_units || (int)c->wptr.size() > kMaxFusedWarps + 1)
    return fail(c, BBC_EINVAL, "internal: warp units exceed their workspace");
  if (!c->ws) return BBC_OK;
  std::vector<int4> wu(c->wunits.size());
  for (size_t i = 0; i < c->wunits.size(); i++)
    wu[i] = make_int4(c->wunits[i].batch, c->wunits[i].side, c->wunits[i].k0, c->wunits[i].k1);
  cudaError_t e = cudaMemcpyAsync(c->d_wptr, c->wptr.data(), sizeof(int) * c->wptr.size(), cudaMemcpyHostToDevice,
                                  c->stream);
  if (e == cudaSuccess && !wu.empty())
    e = cudaMemcpyAsync(c->d_wunits, wu.data(), sizeof(int4) * wu.size(), cudaMemcpyHostToDevice, c->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
  if (e != cudaSuccess) return cuda_fail(c, e, "warp unit upload");
  return BBC_OK;
}

// Average device time of `reps` launches by `launch` on the context stream
// (one untimed launch first).  Returns a negative value on a failed launch.
template <typename F>
double time_launches(bbc_ctx* c, int reps, F launch) {
  if (launch() != cudaSuccess) return -1.0;
  cudaEvent_t a = nullptr, b = nullptr;
  if (cudaEventCreate(&a) != cudaSuccess || cudaEventCreate(&b) != cudaSuccess) {
    if (a) cudaEventDestroy(a);
    return -1.0;
  }
  cudaEventRecord(a, c->stream);
  bool ok = true;
  for (int i = 0; i < reps && ok; i++) ok = launch() == cudaSuccess;
  cudaEventRecord(b, c->stream);
  float ms = -1.f;
  if (ok && cudaEventSynchronize(b) == cudaSuccess) cudaEventElapsedTime(&ms, a, b);
  cudaEventDestroy(a);
  cudaEventDestroy(b);
  return ok && ms >= 0.f ? ms / reps : -1.0;
}

// Sticky record of the bounded device waits (synchronous): BBC_ETIMEOUT, the
// record cleared, if a wait gave up since the last read -- bit 0: the
// queue-driven forward FFT (every slot is then marked unbuilt), bit 1: the
// tensor-core contraction (its correlators are not valid).
bbc_status wait_status(bbc_ctx* c) {
  int err = 0;
  cudaError_t e = cudaMemcpyAsync(&err, c->d_qerr, sizeof(int), cudaMemcpyDeviceToHost, c->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
  if (e != cudaSuccess) return cuda_fail(c, e, "device status");
  if (!err) return BBC_OK;
  e = cudaMemsetAsync(c->d_qerr, 0, sizeof(int), c->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
  if (e != cudaSuccess) return cuda_fail(c, e, "device status");
  if (err & 1) {
    for (auto& b : c->slot_built) b = 0;
    return fail(c, BBC_ETIMEOUT, "a bounded wait of the queue-driven forward FFT gave up: the blocks are not valid");
  }
  return fail(c, BBC_ETIMEOUT,
              "a bounded wait of the tensor-core contraction gave up: the correlators of the last contraction are not "
              "valid");
}

// The block build of slots [0, n_slots): the dense-tuple FP32 kernel, or the
// entry-per-thread kernel (FP64, double-float, and FP32 without dense tables).
cudaError_t launch_build(bbc_ctx* c, int n_slots, int sites, int threads) {
  const bbc::Plan& p = c->plan;
  if (c->dense)
    return bbc::launch_block_build_dense(c->d_prop, c->V, n_slots, c->d_dchunk, c->d_dell, c->d_dtuples,
                                         bbc::dev_groups(p, &c->db), c->d_blk, p.n_out, c->stream, sites, threads);
  return bbc::launch_block_build(c->d_prop, c->V, n_slots, c->d_ell_chunk, c->d_ell, c->d_zneed, bbc::dev_groups(p),
                                 c->d_blk, p.n_out, real_kind(c->prec), c->stream, sites, threads);
}

// The tensor-core contraction of one slot: G(q) of every pair {q, -q} on
// the tensor cores, then the CUDA-core products and the Wick sums.  The
// pairs are cut into chunks: the tensor-core kernel of chunk k + 1 runs on
// the context stream while the CUDA-core kernel of chunk k runs on a second
// stream (forked and joined with events, so a stream capture records the
// same dependencies); the two kernels fill different pipes of the SMs.
cudaError_t launch_tc(bbc_ctx* c, int slot) {
  const bbc::Plan& p = c->plan;
  const char* blk = c->d_blk + (size_t)slot * c->V * p.n_out * cplx_bytes(c->prec);
  const int n_q = (int)c->qlist.size();
  const int g_elems = c->tcs.nbp * c->tcs.nbp;
  const int mode = c->prec == BBC_MIXED_TF32 ? bbc::kTc1x : bbc::kTc3x;
  auto tc = [&](int q0, int q1, cudaStream_t st) {
    if (c->tune.tc_kernel == 0)
      return bbc::launch_contract_umma(blk, c->lat.L, p.n_out, c->d_tc_base, c->tcs.nb, c->tcs.nbp, c->d_qlist + q0,
                                       q1 - q0, c->d_G + (size_t)q0 * g_elems * 8, mode, c->d_qerr,
                                       bbc::kFftSpinLimit, st);
    return bbc::launch_contract_tc(blk, c->lat.L, p.n_out, c->d_tc_base, c->tcs.nb, c->tcs.nbp, c->d_qlist + q0,
                                   q1 - q0, c->d_tc_units, (int)c->tcs.units.size(),
                                   c->d_G + (size_t)q0 * g_elems * 8, mode, st);
  };
  auto rest = [&](int q0, int q1, cudaStream_t st) {
    return bbc::launch_contract_rest(blk, c->lat.L, p.n_out, c->d_row_map, c->tcs.rest.n_out, c->n_slots,
                                     c->d_qlist + q0, q1 - q0, c->d_tasks, (int)c->tcs.rest.tasks.size(),
                                     c->d_batches, c->d_wptr, c->d_wunits, c->d_G + (size_t)q0 * g_elems * 8, g_elems,
                                     c->d_tc_cptr, c->d_tc_terms, c->d_tc_coefs, (int)c->tcs.coef_values.size(),
                                     (int)p.channels.size(), c->d_ct, c->tune.fused_warps, c->tune.fused_steps, st);
  };
  constexpr int K = bbc_ctx::kTcChunks;
  // with fewer pairs (L = 16: 2052) a chunk is about one wave of CTAs and its
  // tail costs more than the overlap gains (measured): one stream there.  The
  // tcgen05 kernel holds every SM's shared memory, so nothing runs beside it:
  // one stream for it too.
  constexpr int kMinPairs = 4096;
  cudaError_t e = cudaSuccess;
  if (c->tune.tc_kernel == 0) {
    e = tc(0, n_q, c->stream);
    return e == cudaSuccess ? rest(0, n_q, c->stream) : e;
  }
  if (n_q >= kMinPairs && !c->side) {  // the second stream and its events, once
    e = cudaStreamCreateWithFlags(&c->side, cudaStreamNonBlocking);
    for (int k = 0; k < K && e == cudaSuccess; k++) e = cudaEventCreateWithFlags(&c->fork[k], cudaEventDisableTiming);
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&c->join, cudaEventDisableTiming);
    if (e != cudaSuccess) return e;
  }
  if (n_q < kMinPairs) {
    e = tc(0, n_q, c->stream);
    return e == cudaSuccess ? rest(0, n_q, c->stream) : e;
  }
  for (int k = 0; k < K && e == cudaSuccess; k++) {
    const int q0 = (int)((long long)n_q * k / K), q1 = (int)((long long)n_q * (k + 1) / K);
    e = tc(q0, q1, c->stream);
    if (e == cudaSuccess) e = cudaEventRecord(c->fork[k], c->stream);
    if (e == cudaSuccess) e = cudaStreamWaitEvent(c->side, c->fork[k], 0);
    if (e == cudaSuccess) e = rest(q0, q1, c->side);
  }
  if (e == cudaSuccess) e = cudaEventRecord(c->join, c->side);
  if (e == cudaSuccess) e = cudaStreamWaitEvent(c->stream, c->join, 0);
  return e;
}

}  // namespace

extern "C" {

bbc_status bbc_create(bbc_ctx** ctx, const bbc_lattice* lat, bbc_precision prec, const int* channels,
                      int n_channels, void* cuda_stream) {
  return bbc_create_components(ctx, lat, prec, channels, n_channels, BBC_UPPER, cuda_stream);
}

bbc_status bbc_create_components(bbc_ctx** ctx, const bbc_lattice* lat, bbc_precision prec, const int* channels,
                                 int n_channels, bbc_components components, void* cuda_stream) {
  if (!ctx || !lat || !channels) return fail(nullptr, BBC_EINVAL, "null argument");
  *ctx = nullptr;
  if (!supported_L(lat->L)) return fail(nullptr, BBC_EINVAL, "unsupported L (supported: 2, 4, 8, 16, 24, 32, 48)");
  if (lat->T < 1 || lat->t0 < 0 || lat->t0 >= lat->T) return fail(nullptr, BBC_EINVAL, "bad T or t0");
  if (prec != BBC_FP64 && prec != BBC_MIXED_FP32 && prec != BBC_MIXED_BF16 && prec != BBC_DF64 &&
      prec != BBC_MIXED_TF32)
    return fail(nullptr, BBC_EINVAL, "bad precision");
  if (n_channels < 1 || n_channels > bbc::kMaxChannels) return fail(nullptr, BBC_EINVAL, "bad channel count");
  if (components != BBC_UPPER && components != BBC_LOWER) return fail(nullptr, BBC_EINVAL, "bad spin components");
  bbc_ctx* c = new (std::nothrow) bbc_ctx();
  if (!c) return fail(nullptr, BBC_ENOMEM, "host allocation failed");
  c->lat = *lat;
  c->prec = prec;
  c->stream = (cudaStream_t)cuda_stream;
  c->V = lat->L * lat->L * lat->L;
  std::string err;
  try {
    if (!bbc::build_plan(channels, n_channels, &c->plan, &err, components == BBC_LOWER ? 2 : 0)) {
      delete c;
      return fail(nullptr, BBC_EINVAL, err);
    }
  } catch (const std::bad_alloc&) {
    delete c;
    return fail(nullptr, BBC_ENOMEM, "host allocation failed while planning");
  } catch (...) {
    delete c;
    return fail(nullptr, BBC_EINVAL, "planner failed");
  }
  // FP32 blocks from dense entry tuples when the tables and shared memory allow
  if (real_kind(prec) == bbc::RK_F32 && c->plan.groups.size() <= (size_t)bbc::kMaxBuildGroups) {
    std::string derr;
    try {
      c->dense = bbc::make_dense_build(c->plan, &c->db, &derr) &&
                 bbc::dense_build_smem(bbc::dev_groups(c->plan, &c->db), 1) <= bbc::kMaxSmemPerBlock;
    } catch (const std::bad_alloc&) {
      c->dense = false;
    }
    if (!c->dense) c->db = bbc::DenseBuild();
  }
  // warp task groups of the pair products: enough warps per 32 q to fill the
  // GPU several times over at L = 16 (V/32 q tiles x groups warps); the
  // double-float products start with more, shorter groups (fewer q tiles in
  // flight, so their rows stay in L2); the autotuner may choose others
  c->tune.pair_groups = prec == BBC_DF64 ? 192 : 48;
  for (int q = 0; q < c->V; q++) {  // one q of every pair {q, -q}
    const int Ls = lat->L, qx = q % Ls, qy = (q / Ls) % Ls, qz = q / (Ls * Ls);
    const int nq = (Ls - qx) % Ls + Ls * ((Ls - qy) % Ls + Ls * ((Ls - qz) % Ls));
    if (q <= nq) c->qlist.push_back(q);
  }
  // tensor cores for the trace-form block pairs (mixed FP32 and TF32): the
  // rest kernel must fit one CTA's shared memory, else the contraction stays
  // on the CUDA cores
  if (tensor_path(prec)) {
    try {
      std::string serr;
      if (!bbc::split_tensor_tasks(c->plan, &c->tcs, &serr)) {
        delete c;
        return fail(nullptr, BBC_EINVAL, serr);
      }
      if (c->tcs.nb > 0) {
        c->tc = true;
        const FusedSchedule& f = fused_schedule(c->plan, c->tcs.rest, true);
        const int n_slots = f.layout.n_slots;
        const int g_elems = c->tcs.nbp * c->tcs.nbp;
        if (bbc::contract_rest_smem(n_slots, (int)c->tcs.rest.tasks.size(), g_elems,
                                    (int)c->tcs.coef_values.size()) > bbc::kMaxSmemPerBlock ||
            c->tcs.rest.n_out > 65536 || n_slots > 65536 || c->plan.n_out > 65536 ||
            2 * 16 * (int)c->tcs.rest.tasks.size() + g_elems > 65536 ||
            bbc::contract_tc_smem(c->tcs.nbp) > bbc::kMaxSmemPerBlock || c->tcs.rest.tasks.empty()) {
          c->tc = false;
          c->tcs = bbc::TcSplit();
        }
      } else {
        c->tcs = bbc::TcSplit();
      }
    } catch (const std::bad_alloc&) {
      delete c;
      return fail(nullptr, BBC_ENOMEM, "host allocation failed while scheduling");
    }
  }
  if (c->tc) {
    const FusedSchedule& f = fused_schedule(c->plan, c->tcs.rest, true);
    c->fused = true;
    c->batches = f.batches;
    c->row_slot = f.layout.row_slot;
    c->n_slots = f.layout.n_slots;
    c->tune.fused_warps = 8;
    c->tune.fused_steps = 1;
    std::vector<int> wp;
    std::vector<bbc::BatchUnit> wu;
    for (int w : kRestWarpsCand)
      for (int k : kChunkCand) {
        bbc::make_units(c->tcs.rest, f.batches, w, k, &wp, &wu);
        c->max_units = std::max(c->max_units, wu.size());
      }
    bool ok = (int)c->row_slot.size() == c->tcs.rest.n_out;
    for (int i = 0; ok && i < c->tcs.rest.n_out; i++)
      ok = c->row_slot[i] >= (i ? c->row_slot[i - 1] + 1 : 0) && c->row_slot[i] < c->n_slots;
    for (size_t i = 0; ok && i < c->tcs.row_src.size(); i++) ok = c->tcs.row_src[i] >= 0 && c->tcs.row_src[i] < c->plan.n_out;
    const int n_v = 2 * 16 * (int)c->tcs.rest.tasks.size() + c->tcs.nbp * c->tcs.nbp;
    for (size_t i = 0; ok && i < c->tcs.src_q.size(); i++)
      ok = c->tcs.src_q[i] >= 0 && c->tcs.src_q[i] < n_v && c->tcs.src_mq[i] >= 0 && c->tcs.src_mq[i] < n_v;
    for (int u : c->tcs.units) {
      if (!ok) break;
      const int mt = u & 0xff, nt0 = (u >> 8) & 0xff, cnt = u >> 16;
      ok = cnt >= 1 && cnt <= bbc::kTcTilesPerWarp && 16 * (mt + 1) <= c->tcs.nbp && 8 * (nt0 + cnt) <= c->tcs.nbp;
    }
    if (!ok) {
      delete c;
      return fail(nullptr, BBC_EINVAL, "internal: tensor-core schedule is not valid");
    }
  }
  // fused FP32 contraction: warp batches, bank layout, one q of every pair {q, -q}
  if (fused_path(prec) && !c->tc) {
    try {
      const FusedSchedule& f = fused_schedule(c->plan, c->plan, false);
      c->batches = f.batches;
      c->row_slot = f.layout.row_slot;
      c->n_slots = f.layout.n_slots;
      std::vector<int> wp;
      std::vector<bbc::BatchUnit> wu;
      for (int w : kFusedWarpsCand)
        for (int k : kChunkCand) {
          bbc::make_units(c->plan, f.batches, w, k, &wp, &wu);
          c->max_units = std::max(c->max_units, wu.size());
        }
    } catch (const std::bad_alloc&) {
      delete c;
      return fail(nullptr, BBC_ENOMEM, "host allocation failed while scheduling");
    }
    // the kernel stages row i at row_slot[i] and reads slot offA + k: slots
    // must be increasing (no two rows share one) and inside n_slots
    bool ok = (int)c->row_slot.size() == c->plan.n_out;
    for (int i = 0; ok && i < c->plan.n_out; i++)
      ok = c->row_slot[i] >= (i ? c->row_slot[i - 1] + 1 : 0) && c->row_slot[i] < c->n_slots;
    if (!ok) {
      delete c;
      return fail(nullptr, BBC_EINVAL, "internal: fused shared-memory layout is not a valid row map");
    }
    c->fused = bbc::contract_fused_smem(c->n_slots, (int)c->plan.tasks.size(), prec == BBC_MIXED_BF16) <=
               bbc::kMaxSmemPerBlock;
    if (!c->fused) {
      if (prec == BBC_MIXED_BF16) {
        delete c;
        return fail(nullptr, BBC_EINVAL,
                    "the bfloat16 trial needs the fused contraction, and this channel list's rows and products "
                    "do not fit one CTA's shared memory: use BBC_MIXED_FP32");
      }
      c->batches.clear();
      c->row_slot.clear();
      c->n_slots = 0;
      c->max_units = 0;
    }
  }
  {  // a configuration tuned earlier in this process for the same problem
    std::lock_guard<std::mutex> lock(g_tune_mutex);
    auto it = g_tuned.find({{lat->L, (int)prec}, plan_key(c->plan)});
    if (it != g_tuned.end()) c->tune = it->second;
  }
  if (apply_fused_units(c) != BBC_OK || apply_pair_groups(c) != BBC_OK) {
    delete c;
    return fail(nullptr, BBC_EINVAL, "internal: warp units or task groups exceed their workspace");
  }
  bbc::cubic_orbits(lat->L, c->orb_ptr, c->orb_site);
  {  // the kernel indexes sites through this table: it must be a partition of the lattice
    std::vector<char> hit(c->V, 0);
    bool ok = c->orb_ptr.front() == 0 && c->orb_ptr.back() == c->V && (int)c->orb_site.size() == c->V;
    for (size_t k = 0; ok && k + 1 < c->orb_ptr.size(); k++)
      ok = c->orb_ptr[k + 1] > c->orb_ptr[k] && c->orb_ptr[k + 1] - c->orb_ptr[k] <= 24;
    for (int s : c->orb_site) {
      if (!ok) break;
      ok = s >= 0 && s < c->V && !hit[s];
      if (ok) hit[s] = 1;
    }
    if (!ok) {
      delete c;
      return fail(nullptr, BBC_EINVAL, "internal: cubic orbit table is not a partition of the lattice");
    }
  }
  *ctx = c;
  return BBC_OK;
}

bbc_status bbc_workspace_size(const bbc_ctx* ctx, int slices, size_t* bytes) {
  if (!ctx || !bytes || slices < 1) return BBC_EINVAL;
  *bytes = layout(ctx, slices).total;
  return BBC_OK;
}

bbc_status bbc_set_workspace(bbc_ctx* c, void* dev_ptr, size_t bytes, int slices) {
  if (!c) return BBC_EINVAL;
  if (!dev_ptr || slices < 1) return fail(c, BBC_EINVAL, "null workspace or slices < 1");
  if (((uintptr_t)dev_ptr) & 255) return fail(c, BBC_EINVAL, "workspace must be 256-byte aligned");
  Layout L = layout(c, slices);
  if (bytes < L.total) return fail(c, BBC_ENOMEM, "workspace too small: need " + std::to_string(L.total) + " bytes");
  if (!c->twiddles) {
    cudaError_t e = bbc::upload_twiddles();
    if (e != cudaSuccess) return cuda_fail(c, e, "twiddle upload");
    c->twiddles = true;
  }
  char* w = (char*)dev_ptr;
  c->ws = w;
  c->ws_bytes = bytes;
  c->slots = slices;
  c->d_ell_chunk = (int2*)(w + L.ell_chunk);
  c->d_ell = (uint32_t*)(w + L.ell);
  c->d_zneed = (uint32_t*)(w + L.zneed);
  c->d_tasks = (bbc::DevTask*)(w + L.tasks);
  c->d_group_ptr = (int*)(w + L.group_ptr);
  c->d_group_task = (int*)(w + L.group_task);
  c->d_cptr = (int*)(w + L.cptr);
  c->d_citem = (int*)(w + L.citem);
  c->d_ccoef = (double*)(w + L.ccoef);
  c->d_ccoef_df = (float2*)(w + L.ccoef_df);
  c->d_batches = (bbc::WarpBatch*)(w + L.batches);
  c->d_wptr = (int*)(w + L.wptr);
  c->d_wunits = (int4*)(w + L.wunits);
  c->d_qlist = (int*)(w + L.qlist);
  c->d_row_slot = (int*)(w + L.row_slot);
  c->d_orb_ptr = (int*)(w + L.orb_ptr);
  c->d_orb_site = (int*)(w + L.orb_site);
  c->d_tc_base = (int*)(w + L.tc_base);
  c->d_tc_units = (int*)(w + L.tc_units);
  c->d_row_map = (uint32_t*)(w + L.row_map);
  c->d_tc_cptr = (int*)(w + L.tc_cptr);
  c->d_tc_terms = (uint2*)(w + L.tc_terms);
  c->d_tc_coefs = (float2*)(w + L.tc_coefs);
  c->d_dtuples = (uint32_t*)(w + L.dtuples);
  c->d_dchunk = (int2*)(w + L.dchunk);
  c->d_dell = (uint32_t*)(w + L.dell);
  c->d_G = c->tc ? w + L.G : nullptr;
  c->d_stage = w + L.stage;
  c->d_prop = w + L.prop;
  c->d_amax = (unsigned long long*)(w + L.amax);
  c->d_kexp = (int*)(w + L.kexp);
  c->d_blk = w + L.blk;
  c->d_blk16 = w + L.blk16;
  c->d_blkf = w + L.blkf;
  c->d_blks = c->prec == BBC_FP64 ? (double*)(w + L.blks) : nullptr;
  c->d_P = w + L.P;
  c->d_ct = w + L.ct;
  c->d_scale = (double*)(w + L.scale);
  c->d_flag = (int*)(w + L.flag);
  c->d_qerr = (int*)(w + L.qerr);
  c->d_fftq = queue_fft(c) ? (int*)(w + L.fftq) : nullptr;
  const bbc::Plan& p = c->plan;
  // the fused kernels address their shared-memory copy of the rows (slots)
  const std::vector<bbc::PairTask>& run_tasks = fused_plan(c).tasks;
  std::vector<bbc::DevTask> tasks(run_tasks.size());
  bbc::to_dev_tasks(run_tasks.data(), run_tasks.size(), c->fused ? &c->row_slot : nullptr, tasks.data());
  // tensor-core path: compact rows (block row | slot << 16), Wick terms and
  // their distinct coefficients split into two FP32 words
  std::vector<uint32_t> row_map(c->tcs.row_src.size());
  for (size_t i = 0; i < row_map.size(); i++) row_map[i] = (uint32_t)c->tcs.row_src[i] | ((uint32_t)c->row_slot[i] << 16);
  std::vector<uint2> tc_terms(c->tcs.coef.size());
  for (size_t i = 0; i < tc_terms.size(); i++)
    tc_terms[i] = make_uint2((uint32_t)c->tcs.src_q[i] | ((uint32_t)c->tcs.src_mq[i] << 16), (uint32_t)c->tcs.coef_index[i]);
  std::vector<float2> tc_coefs;
  for (double x : c->tcs.coef_values) {
    const float h = (float)x;
    tc_coefs.push_back(make_float2(h, (float)(x - (double)h)));
  }
  std::vector<float2> coef_df;  // double-float split of the Wick coefficients
  if (c->prec == BBC_DF64)
    for (double x : p.tcontrib_coef) {
      const float h = (float)x;
      coef_df.push_back(make_float2(h, (float)(x - (double)h)));
    }
  std::vector<bbc::WarpBatch> wb(c->batches.size());
  for (size_t i = 0; i < c->batches.size(); i++) {
    wb[i].n = (int)c->batches[i].tasks.size();
    wb[i].nA = c->batches[i].nA;
    for (int j = 0; j < 32; j++) wb[i].task[j] = j < wb[i].n ? c->batches[i].tasks[j] : 0;
  }
  struct Up { void* dst; const void* src; size_t n; } ups[] = {
      {c->d_ell_chunk, p.ell_chunk.data(), sizeof(int2) * p.ell_chunk.size()},
      {c->d_ell, p.ell.data(), sizeof(uint32_t) * p.ell.size()},
      {c->d_zneed, p.zneed.data(), sizeof(uint32_t) * p.zneed.size()},
      {c->d_tasks, tasks.data(), sizeof(bbc::DevTask) * tasks.size()},
      {c->d_group_ptr, c->group_ptr.data(), sizeof(int) * c->group_ptr.size()},
      {c->d_group_task, c->group_task.data(), sizeof(int) * c->group_task.size()},
      {c->d_cptr, p.tcontrib_ptr.data(), sizeof(int) * p.tcontrib_ptr.size()},
      {c->d_citem, p.tcontrib_item.data(), sizeof(int) * p.tcontrib_item.size()},
      {c->d_ccoef, p.tcontrib_coef.data(), sizeof(double) * p.tcontrib_coef.size()},
      {c->d_ccoef_df, coef_df.data(), sizeof(float2) * coef_df.size()},
      {c->d_batches, wb.data(), sizeof(bbc::WarpBatch) * wb.size()},
      {c->d_qlist, c->qlist.data(), sizeof(int) * c->qlist.size()},
      {c->d_row_slot, c->row_slot.data(), sizeof(int) * c->row_slot.size()},
      {c->d_orb_ptr, c->orb_ptr.data(), sizeof(int) * c->orb_ptr.size()},
      {c->d_orb_site, c->orb_site.data(), sizeof(int) * c->orb_site.size()},
      {c->d_tc_base, c->tcs.base.data(), sizeof(int) * c->tcs.base.size()},
      {c->d_tc_units, c->tcs.units.data(), sizeof(int) * c->tcs.units.size()},
      {c->d_row_map, row_map.data(), sizeof(uint32_t) * row_map.size()},
      {c->d_tc_cptr, c->tcs.out_ptr.data(), sizeof(int) * c->tcs.out_ptr.size()},
      {c->d_tc_terms, tc_terms.data(), sizeof(uint2) * tc_terms.size()},
      {c->d_tc_coefs, tc_coefs.data(), sizeof(float2) * tc_coefs.size()},
      {c->d_dtuples, c->db.tuples.data(), sizeof(uint32_t) * c->db.tuples.size()},
      {c->d_dchunk, c->db.ell_chunk.data(), sizeof(int2) * c->db.ell_chunk.size()},
      {c->d_dell, c->db.ell.data(), sizeof(uint32_t) * c->db.ell.size()},
  };
  cudaError_t e0 = cudaMemsetAsync(c->d_qerr, 0, sizeof(int), c->stream);
  if (e0 != cudaSuccess) return cuda_fail(c, e0, "workspace status word");
  for (auto& u : ups) {
    if (u.n == 0) continue;
    // synchronous copy from pageable host memory: the tables are live only
    // as long as this call
    cudaError_t e = cudaMemcpyAsync(u.dst, u.src, u.n, cudaMemcpyHostToDevice, c->stream);
    if (e != cudaSuccess) return cuda_fail(c, e, "table upload");
  }
  cudaError_t e = cudaStreamSynchronize(c->stream);
  if (e != cudaSuccess) return cuda_fail(c, e, "table upload");
  c->slot_t.assign(slices, -1);
  c->slot_loaded.assign(slices, 0);
  c->slot_built.assign(slices, 0);
  return apply_fused_units(c);
}

bbc_status bbc_load_propagator(bbc_ctx* c, int flavour, int slot, int t, const void* data, int dtype,
                               int on_device) {
  if (!c) return BBC_EINVAL;
  if (!c->ws) return fail(c, BBC_ESTATE, "no workspace attached");
  if (flavour != BBC_LIGHT && flavour != BBC_STRANGE) return fail(c, BBC_EINVAL, "bad flavour");
  if (slot < 0 || slot >= c->slots) return fail(c, BBC_EINVAL, "bad slot");
  if (t < 0 || t >= c->lat.T) return fail(c, BBC_EINVAL, "bad time slice");
  if (!data) return fail(c, BBC_EINVAL, "null propagator");
  if (dtype != BBC_C128 && dtype != BBC_C64) return fail(c, BBC_EINVAL, "bad dtype");
  const size_t nc = (size_t)c->V * 144;
  const size_t in_bytes = nc * (dtype == BBC_C128 ? 16 : 8);
  const void* src = data;
  if (!on_device) {
    char* stage = c->d_stage + ((size_t)slot * 2 + flavour) * nc * 16;
    cudaError_t e = cudaMemcpyAsync(stage, data, in_bytes, cudaMemcpyHostToDevice, c->stream);
    if (e != cudaSuccess) return cuda_fail(c, e, "propagator upload");
    src = stage;
  } else if (((uintptr_t)data) & 15) {
    return fail(c, BBC_EINVAL, "device propagator must be 16-byte aligned");
  }
  unsigned long long* amax = c->d_amax + slot * 2 + flavour;
  int* kexp = c->d_kexp + slot * 2 + flavour;
  StageScope scope(c, BBC_STAGE_INGEST);
  cudaError_t e = cudaMemsetAsync(amax, 0, sizeof(*amax), c->stream);
  if (e != cudaSuccess) return cuda_fail(c, e, "memset");
  e = bbc::launch_absmax(src, dtype, (long long)nc, amax, c->stream);
  if (e != cudaSuccess) return cuda_fail(c, e, "absmax kernel");
  char* dst = c->d_prop + ((size_t)slot * 2 + flavour) * nc * cplx_bytes(c->prec);
  e = bbc::launch_convert(src, dtype, (long long)nc, amax, kexp, dst, real_kind(c->prec), c->stream);
  if (e != cudaSuccess) return cuda_fail(c, e, "convert kernel");
  if (c->checks & BBC_CHECK_INPUT) {
    unsigned long long bits = 0;
    e = cudaMemcpyAsync(&bits, amax, sizeof(bits), cudaMemcpyDeviceToHost, c->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
    if (e != cudaSuccess) return cuda_fail(c, e, "input check");
    if (bits >= 0x7ff0000000000000ull)
      return fail(c, BBC_ENUMERIC, std::string(flavour == BBC_LIGHT ? "light" : "strange") +
                                       " propagator of slice " + std::to_string(t) + " has a NaN or infinite entry");
  }
  if (c->slot_t[slot] != t) {
    c->slot_loaded[slot] = 0;
    c->slot_t[slot] = t;
  }
  c->slot_loaded[slot] |= 1 << flavour;
  c->slot_built[slot] = 0;
  return BBC_OK;
}

bbc_status bbc_build_blocks(bbc_ctx* c, int n_slots) {
  if (!c) return BBC_EINVAL;
  if (!c->ws) return fail(c, BBC_ESTATE, "no workspace attached");
  if (n_slots < 1 || n_slots > c->slots) return fail(c, BBC_EINVAL, "bad slot count");
  for (int s = 0; s < n_slots; s++)
    if (c->slot_loaded[s] != 3) return fail(c, BBC_ESTATE, "slot " + std::to_string(s) + " lacks a propagator");
  const bool fp64 = fp64_storage(c->prec);
  const bbc::Plan& p = c->plan;
  cudaError_t e;
  {
    StageScope scope(c, BBC_STAGE_BUILD);
    e = launch_build(c, n_slots, c->tune.build_sites, c->tune.build_threads);
    if (e != cudaSuccess) return cuda_fail(c, e, "block build");
  }
  {
    StageScope scope(c, BBC_STAGE_FFT_FWD);
    // FP64 and unfused FP32: field-major copy for the lanes-over-q products;
    // fused FP32: in place, q-major
    e = c->prec == BBC_DF64 ? bbc::launch_fft_forward_df(c->d_blk, c->d_blkf, c->lat.L, n_slots, p.n_out, c->stream)
        : !c->fused         ? bbc::launch_fft_forward(c->d_blk, c->d_blkf, c->lat.L, n_slots, p.n_out, fp64, c->stream,
                                                      c->d_blks)
        : queue_fft(c)      ? bbc::launch_fft_forward_queue(c->d_blk, c->lat.L, n_slots, p.n_out,
                                                        bbc::FftQueue{c->d_fftq, c->d_qerr}, -1, bbc::kFftSpinLimit,
                                                        c->stream)
                            : bbc::launch_fft_forward_site(c->d_blk, c->lat.L, n_slots, p.n_out, fp64, c->stream);
    if (e != cudaSuccess) return cuda_fail(c, e, "forward FFT");
    if (c->prec == BBC_MIXED_BF16) {
      e = bbc::launch_to_bf16(c->d_blk, c->d_blk16, (size_t)n_slots * c->V * p.n_out, c->stream);
      if (e != cudaSuccess) return cuda_fail(c, e, "bfloat16 rounding");
    }
  }
  for (int s = 0; s < n_slots; s++) c->slot_built[s] = 1;
  return BBC_OK;
}

bbc_status bbc_contract(bbc_ctx* c, int slot, void* out_dev, int normalised) {
  if (!c) return BBC_EINVAL;
  if (!c->ws) return fail(c, BBC_ESTATE, "no workspace attached");
  if (slot < 0 || slot >= c->slots) return fail(c, BBC_EINVAL, "bad slot");
  if (!c->slot_built[slot]) return fail(c, BBC_ESTATE, "blocks of this slot are not built");
  if (!out_dev || (((uintptr_t)out_dev) & 15)) return fail(c, BBC_EINVAL, "output must be a 16-byte aligned device pointer");
  const bool fp64 = fp64_storage(c->prec);
  const bbc::Plan& p = c->plan;
  const int n_ch = (int)p.channels.size();
  cudaError_t e;
  if (!c->fused) {
    const char* blkf = c->d_blkf + (size_t)slot * c->V * p.n_out * cplx_bytes(c->prec);
    const double* blks = c->d_blks ? c->d_blks + (size_t)slot * c->V * p.n_out : nullptr;
    {
      StageScope scope(c, BBC_STAGE_CONTRACT);
      e = c->prec == BBC_DF64
              ? bbc::launch_pair_products_df(blkf, c->lat.L, c->d_tasks, c->d_group_ptr, c->d_group_task,
                                             (int)c->group_ptr.size() - 1, c->d_P, c->stream)
              : bbc::launch_pair_products(blkf, c->lat.L, c->d_tasks, c->d_group_ptr, c->d_group_task,
                                          (int)c->group_ptr.size() - 1, c->d_P, fp64, c->stream, blks);
      if (e != cudaSuccess) return cuda_fail(c, e, "pair products");
    }
    {
      StageScope scope(c, BBC_STAGE_WICK);
      e = c->prec == BBC_DF64
              ? bbc::launch_wick_sums_df(c->d_P, c->lat.L, c->d_cptr, c->d_citem, c->d_ccoef_df, n_ch, c->d_ct,
                                         c->stream)
              : bbc::launch_wick_sums(c->d_P, c->lat.L, c->d_cptr, c->d_citem, c->d_ccoef, n_ch, c->d_ct, fp64,
                                      c->stream);
      if (e != cudaSuccess) return cuda_fail(c, e, "Wick sums");
    }
  } else if (c->tc) {
    StageScope scope(c, BBC_STAGE_CONTRACT);
    e = launch_tc(c, slot);
    if (e != cudaSuccess) return cuda_fail(c, e, "tensor-core contraction");
  } else {
    const bool bf16 = c->prec == BBC_MIXED_BF16;
    const char* blk = bf16 ? c->d_blk16 + (size_t)slot * c->V * p.n_out * 4
                           : c->d_blk + (size_t)slot * c->V * p.n_out * cplx_bytes(c->prec);
    StageScope scope(c, BBC_STAGE_CONTRACT);
    e = bbc::launch_contract_fused(blk, c->lat.L, p.n_out, c->d_row_slot, c->n_slots, c->d_qlist,
                                   (int)c->qlist.size(), c->d_tasks,
                                   (int)p.tasks.size(), c->d_batches, c->d_wptr, c->d_wunits, c->d_cptr, c->d_citem,
                                   c->d_ccoef, n_ch, c->d_ct, c->tune.fused_warps, c->tune.fused_steps, bf16,
                                   c->stream);
    if (e != cudaSuccess) return cuda_fail(c, e, "fused contraction");
  }
  bbc::ScaleParams sp{};
  sp.n_ch = n_ch;
  const int t = c->slot_t[slot];
  const int d = time_distance(c, t);
  for (int i = 0; i < n_ch; i++) {
    const int ns = p.n_strange[i];
    const double mass = (6 - ns) * c->lat.m_ud + ns * c->lat.m_s;  // m_B1 + m_B2
    sp.f[i] = (1.0 / c->V) * (normalised ? std::exp(mass * d) : 1.0);
    sp.nl[i] = 6 - ns;
    sp.ns[i] = ns;
  }
  {
    StageScope scope(c, BBC_STAGE_NORMALISE);
    e = bbc::launch_scales(sp, c->d_kexp + slot * 2, c->d_scale, c->stream);
    if (e != cudaSuccess) return cuda_fail(c, e, "normalisation");
  }
  {
    StageScope scope(c, BBC_STAGE_FFT_INV);
    e = c->prec == BBC_DF64 ? bbc::launch_fft_inverse_df(c->d_ct, out_dev, c->lat.L, n_ch, c->d_scale, c->stream)
        : !c->fused ? bbc::launch_fft_inverse(c->d_ct, out_dev, c->lat.L, n_ch, c->d_scale, fp64, c->stream)
               : bbc::launch_fft_inverse_site(c->d_ct, out_dev, c->lat.L, n_ch, c->d_scale, fp64, c->stream, c->tc);
    if (e != cudaSuccess) return cuda_fail(c, e, "inverse FFT");
  }
  if (c->checks & BBC_CHECK_OUTPUT) {
    int flag = 0;
    e = cudaMemsetAsync(c->d_flag, 0, sizeof(int), c->stream);
    if (e == cudaSuccess)
      e = bbc::launch_nonfinite((const double*)out_dev, (long long)n_ch * c->V * 32, c->d_flag, c->stream);
    if (e == cudaSuccess) e = cudaMemcpyAsync(&flag, c->d_flag, sizeof(int), cudaMemcpyDeviceToHost, c->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
    if (e != cudaSuccess) return cuda_fail(c, e, "output check");
    const bbc_status ws = wait_status(c);  // a timed-out FFT wait explains any output
    if (ws != BBC_OK) return ws;
    if (flag) return fail(c, BBC_ENUMERIC, "correlators of slice " + std::to_string(t) + " have a NaN or infinite entry");
  }
  return BBC_OK;
}

bbc_status bbc_device_status(bbc_ctx* c) {
  if (!c) return BBC_EINVAL;
  if (!c->ws) return BBC_OK;  // nothing has run
  return wait_status(c);
}

bbc_status bbc_check_bounded_wait(bbc_ctx* c, long long spin_limit) {
  if (!c) return BBC_EINVAL;
  if (spin_limit < 1 || spin_limit > bbc::kFftSpinLimit) return fail(c, BBC_EINVAL, "spin_limit outside [1, 2^22]");
  if (!c->ws) return fail(c, BBC_ESTATE, "no workspace attached");
  if (!queue_fft(c)) return fail(c, BBC_ESTATE, "this context has no queue-driven forward FFT");
  // a dependency count of L + 1 planes: no line unit's wait can end
  cudaError_t e = bbc::launch_fft_forward_queue(c->d_blk, c->lat.L, 1, c->plan.n_out,
                                                bbc::FftQueue{c->d_fftq, c->d_qerr}, c->lat.L + 1, spin_limit,
                                                c->stream);
  if (e != cudaSuccess) return cuda_fail(c, e, "bounded-wait self-test");
  return wait_status(c);
}

bbc_status bbc_batch_run(const bbc_batch_item* items, int n_items, void* cuda_stream, int* failed_item) {
  if (failed_item) *failed_item = -1;
  if (!items || n_items < 1) return fail(nullptr, BBC_EINVAL, "empty batch");
  const cudaStream_t st = (cudaStream_t)cuda_stream;
  for (int i0 = 0; i0 < n_items;) {
    bbc_ctx* c = items[i0].ctx;
    if (!c) {
      if (failed_item) *failed_item = i0;
      return fail(nullptr, BBC_EINVAL, "batch item " + std::to_string(i0) + " has no context");
    }
    // a wave: the consecutive items of this context, up to its slot count
    const int cap = std::max(1, c->slots);
    int n = 1;
    while (n < cap && i0 + n < n_items && items[i0 + n].ctx == c) n++;
    const cudaStream_t own = c->stream;
    c->stream = st;
    bbc_status s = BBC_OK;
    int bad = i0;
    for (int j = 0; j < n && s == BBC_OK; j++) {
      const bbc_batch_item& it = items[i0 + j];
      bad = i0 + j;
      s = bbc_load_propagator(c, BBC_LIGHT, j, it.t, it.S_light, it.dtype, it.on_device);
      if (s == BBC_OK) s = bbc_load_propagator(c, BBC_STRANGE, j, it.t, it.S_strange, it.dtype, it.on_device);
    }
    if (s == BBC_OK) {
      bad = i0;
      s = bbc_build_blocks(c, n);  // one block build and one forward FFT over the wave's slots
    }
    for (int j = 0; j < n && s == BBC_OK; j++) {
      const bbc_batch_item& it = items[i0 + j];
      bad = i0 + j;
      s = bbc_contract(c, j, it.out_dev, it.normalised);
    }
    c->stream = own;
    if (s != BBC_OK) {
      if (failed_item) *failed_item = bad;
      return s;
    }
    i0 += n;
  }
  return BBC_OK;
}

bbc_status bbc_set_checks(bbc_ctx* c, int flags) {
  if (!c) return BBC_EINVAL;
  if (flags & ~(BBC_CHECK_INPUT | BBC_CHECK_OUTPUT)) return fail(c, BBC_EINVAL, "unknown check flags");
  c->checks = flags;
  return BBC_OK;
}

bbc_status bbc_get_tuning(const bbc_ctx* c, bbc_tuning* t) {
  if (!c || !t) return BBC_EINVAL;
  *t = c->tune;
  return BBC_OK;
}

bbc_status bbc_set_tuning(bbc_ctx* c, const bbc_tuning* t) {
  if (!c || !t) return BBC_EINVAL;
  bbc_tuning want = *t;
  if (!c->fused) {  // the FP64 and unfused FP32 paths have no fused kernel to configure
    want.fused_warps = c->tune.fused_warps;
    want.fused_chunk = c->tune.fused_chunk;
    want.fused_steps = c->tune.fused_steps;
  } else {  // and the fused kernel has no pair-product task lists
    want.pair_groups = c->tune.pair_groups;
  }
  if (!c->tc) want.tc_kernel = c->tune.tc_kernel;  // no tensor-core kernel to choose
  if (!tuning_valid(c, want)) return fail(c, BBC_EINVAL, "unsupported launch configuration");
  const bbc_tuning old = c->tune;
  c->tune = want;
  bbc_status st = apply_fused_units(c);
  if (st == BBC_OK) st = apply_pair_groups(c);
  if (st != BBC_OK) {
    c->tune = old;
    apply_fused_units(c);
    apply_pair_groups(c);
  }
  return st;
}

bbc_status bbc_autotune(bbc_ctx* c, int reps, bbc_tuning* best, double* ms, int cap, int* n_tried) {
  if (!c) return BBC_EINVAL;
  if (reps < 1 || reps > 1000) return fail(c, BBC_EINVAL, "reps must be in [1, 1000]");
  if (!c->ws) return fail(c, BBC_ESTATE, "no workspace attached");
  if (c->slot_loaded[0] != 3) return fail(c, BBC_ESTATE, "slot 0 needs both propagators loaded");
  const bbc::Plan& p = c->plan;
  int n = 0;
  auto record = [&](double v) {
    if (ms && n < cap) ms[n] = v;
    n++;
  };
  // block build: sites per CTA and threads
  bbc_tuning t = c->tune;
  double best_ms = -1.0;
  for (const auto& bc : kBuildCand) {
    bbc_tuning cand = c->tune;
    cand.build_sites = bc[0];
    cand.build_threads = bc[1];
    if (!tuning_valid(c, cand)) { record(-1.0); continue; }
    const double v = time_launches(c, reps, [&] { return launch_build(c, 1, bc[0], bc[1]); });
    record(v);
    if (v < 0) return cuda_fail(c, cudaGetLastError(), "autotune: block build");
    if (best_ms < 0 || v < best_ms) { best_ms = v; t.build_sites = bc[0]; t.build_threads = bc[1]; }
  }
  c->tune.build_sites = t.build_sites;
  c->tune.build_threads = t.build_threads;
  // slot 0 rebuilt with the chosen configuration (blocks and forward FFT)
  c->slot_built[0] = 0;
  bbc_status st = bbc_build_blocks(c, 1);
  if (st != BBC_OK) return st;
  if (c->fused) {  // fused contraction: warps per CTA and open-index chunk per warp unit
    const bool bf16 = c->prec == BBC_MIXED_BF16;
    const char* blk = bf16 ? c->d_blk16 : c->d_blk;
    best_ms = -1.0;
    const std::vector<int> warps_cand = c->tc ? std::vector<int>(std::begin(kRestWarpsCand), std::end(kRestWarpsCand))
                                              : std::vector<int>(std::begin(kFusedWarpsCand), std::end(kFusedWarpsCand));
    for (int wv : warps_cand)
      for (int sv : kFusedStepsCand) {
        if (c->tc ? !bbc::rest_variant_supported(wv, sv) : !bbc::fused_variant_supported(wv, sv)) continue;
        for (int kv : kChunkCand) {
          c->tune.fused_warps = wv;
          c->tune.fused_steps = sv;
          c->tune.fused_chunk = kv;
          st = apply_fused_units(c);
          if (st != BBC_OK) return st;
          const double v = time_launches(c, reps, [&] {
            if (c->tc) return launch_tc(c, 0);
            return bbc::launch_contract_fused(blk, c->lat.L, p.n_out, c->d_row_slot, c->n_slots, c->d_qlist,
                                              (int)c->qlist.size(), c->d_tasks, (int)p.tasks.size(), c->d_batches,
                                              c->d_wptr, c->d_wunits, c->d_cptr, c->d_citem, c->d_ccoef,
                                              (int)p.channels.size(), c->d_ct, wv, sv, bf16, c->stream);
          });
          record(v);
          if (v < 0) return cuda_fail(c, cudaGetLastError(), "autotune: fused contraction");
          if (best_ms < 0 || v < best_ms) { best_ms = v; t.fused_warps = wv; t.fused_steps = sv; t.fused_chunk = kv; }
        }
      }
    c->tune.fused_warps = t.fused_warps;
    c->tune.fused_steps = t.fused_steps;
    c->tune.fused_chunk = t.fused_chunk;
    st = apply_fused_units(c);
    if (st != BBC_OK) return st;
    if (c->tc) {  // the trace-form products: tcgen05 or mma.sync (with its two-stream pipeline)
      best_ms = -1.0;
      for (int kv = 0; kv < 2; kv++) {
        c->tune.tc_kernel = kv;
        const double v = time_launches(c, reps, [&] { return launch_tc(c, 0); });
        record(v);
        if (v < 0) return cuda_fail(c, cudaGetLastError(), "autotune: tensor-core kernel");
        if (best_ms < 0 || v < best_ms) { best_ms = v; t.tc_kernel = kv; }
      }
      c->tune.tc_kernel = t.tc_kernel;
    }
  } else {  // block-pair products: task lists per 32 q
    const bool fp64 = fp64_storage(c->prec);
    const double* blks = c->d_blks;
    best_ms = -1.0;
    for (int gv : kPairGroupsCand) {
      c->tune.pair_groups = gv;
      st = apply_pair_groups(c);
      if (st != BBC_OK) return st;
      const int n_groups = (int)c->group_ptr.size() - 1;
      const double v = time_launches(c, reps, [&] {
        return c->prec == BBC_DF64
                   ? bbc::launch_pair_products_df(c->d_blkf, c->lat.L, c->d_tasks, c->d_group_ptr, c->d_group_task,
                                                  n_groups, c->d_P, c->stream)
                   : bbc::launch_pair_products(c->d_blkf, c->lat.L, c->d_tasks, c->d_group_ptr, c->d_group_task,
                                               n_groups, c->d_P, fp64, c->stream, blks);
      });
      record(v);
      if (v < 0) return cuda_fail(c, cudaGetLastError(), "autotune: pair products");
      if (best_ms < 0 || v < best_ms) { best_ms = v; t.pair_groups = gv; }
    }
    c->tune.pair_groups = t.pair_groups;
    st = apply_pair_groups(c);
    if (st != BBC_OK) return st;
  }
  {
    std::lock_guard<std::mutex> lock(g_tune_mutex);
    g_tuned[{{c->lat.L, c->prec}, plan_key(p)}] = c->tune;
  }
  if (best) *best = c->tune;
  if (n_tried) *n_tried = n;
  return BBC_OK;
}

bbc_status bbc_project(bbc_ctx* c, const void* C_dev, int n_fields, void* R_dev, void* Ra1_dev) {
  if (!c) return BBC_EINVAL;
  if (n_fields < 0 || n_fields > 65535) return fail(c, BBC_EINVAL, "n_fields must be in [0, 65535]");
  if (!C_dev || (!R_dev && !Ra1_dev)) return fail(c, BBC_EINVAL, "need an input and at least one output");
  if (((uintptr_t)C_dev | (uintptr_t)R_dev | (uintptr_t)Ra1_dev) & 15)
    return fail(c, BBC_EINVAL, "pointers must be 16-byte aligned");
  const size_t n = (size_t)n_fields * c->V * 16 * 16;
  auto overlap = [n](const void* a, const void* b) {
    if (!a || !b) return false;
    const uintptr_t x = (uintptr_t)a, y = (uintptr_t)b;
    return x < y + n && y < x + n;
  };
  if (overlap(C_dev, R_dev) || overlap(C_dev, Ra1_dev) || overlap(R_dev, Ra1_dev))
    return fail(c, BBC_EINVAL, "input and outputs must not overlap");
  StageScope scope(c, BBC_STAGE_PROJECT);
  if (!c->ws) return fail(c, BBC_ESTATE, "no workspace attached");
  cudaError_t e = bbc::launch_project(C_dev, c->lat.L, c->d_orb_ptr, c->d_orb_site, (int)c->orb_ptr.size() - 1,
                                      n_fields, R_dev, Ra1_dev, c->stream);
  if (e != cudaSuccess) return cuda_fail(c, e, "projection");
  return BBC_OK;
}

bbc_status bbc_plan_stats(const bbc_ctx* c, int channel_pos, int term3, int term4, int* n_diagrams,
                          int* iters_signed, int cap) {
  if (!c || !n_diagrams) return BBC_EINVAL;
  if (channel_pos < 0 || channel_pos >= (int)c->plan.channels.size()) return BBC_EINVAL;
  int n = 0;
  for (const auto& d : c->plan.diagrams)
    if (d.ch_pos == channel_pos && d.term3 == term3 && d.term4 == term4) {
      if (iters_signed && n < cap) iters_signed[n] = d.K * d.parity;
      n++;
    }
  *n_diagrams = n;
  return BBC_OK;
}

bbc_status bbc_plan_sizes(const bbc_ctx* c, int* n_blocks, int* n_block_outputs, int* n_pair_items,
                          long long* pair_macs_per_site) {
  if (!c) return BBC_EINVAL;
  if (n_blocks) *n_blocks = c->plan.n_blocks;
  if (n_block_outputs) *n_block_outputs = c->plan.n_out;
  if (n_pair_items) *n_pair_items = 16 * (int)c->plan.tasks.size();
  if (pair_macs_per_site) *pair_macs_per_site = c->plan.pair_macs;
  return BBC_OK;
}

bbc_status bbc_plan_export(const bbc_ctx* c, int* sizes, int* row_ptr, int* terms, int* tasks, int* out_ptr,
                           int* items, double* coefs) {
  if (!c || !sizes) return BBC_EINVAL;
  const bbc::Plan& p = c->plan;
  const int need[5] = {p.n_out, (int)p.entries.size(), (int)p.tasks.size(), (int)p.tcontrib_item.size(),
                       (int)p.tcontrib_ptr.size() - 1};
  const bool fill = row_ptr && terms && tasks && out_ptr && items && coefs;
  bool fits = true;
  for (int i = 0; i < 5; i++) {
    if (fill && sizes[i] < need[i]) fits = false;  // the caller's capacities
    sizes[i] = need[i];
  }
  if (!fill) return BBC_OK;
  if (!fits) return fail(c, BBC_EINVAL, "plan export: an array is smaller than the plan needs");
  // the tensor entry behind each shared-memory position, group by group, as
  // the build kernel lays them out: a group's zneed list fills positions,
  // and positions of a slot whose family is unchanged carry over
  std::vector<int> pos_slot(8192, -1), pos_local(8192, -1);
  int prev_fam[2] = {-1, -1};
  try {
    for (size_t g = 0; g < p.groups.size(); g++) {
      const bbc::GroupInfo& gi = p.groups[g];
      for (int sl = 0; sl < 2; sl++)
        if (gi.fam[sl] != prev_fam[sl])
          for (int k = 0; k < 8192; k++)
            if (pos_slot[k] == sl) pos_slot[k] = -1;
      for (int z = p.zneed_first[g]; z < p.zneed_first[g + 1]; z++) {
        const uint32_t zn = p.zneed[z];
        const int pos = (int)(zn & 0x1fff);
        pos_slot[pos] = (int)((zn >> 13) & 1);
        pos_local[pos] = (int)(zn >> 14);
      }
      for (int r = gi.first_row; r < gi.first_row + gi.n_rows; r++)
        for (int k = p.row_ptr[r]; k < p.row_ptr[r + 1]; k++) {
          const uint32_t e = p.entries[k];
          const int pos = (int)(e & 0xffff);
          if (pos >= 8192 || pos_slot[pos] < 0 || gi.fam[pos_slot[pos]] < 0)
            return fail(c, BBC_EINVAL, "internal: plan position");
          terms[3 * k] = gi.fam[pos_slot[pos]];
          terms[3 * k + 1] = pos_local[pos];
          terms[3 * k + 2] = (int)(int16_t)(e >> 16);
        }
      prev_fam[0] = gi.fam[0];
      prev_fam[1] = gi.fam[1];
    }
  } catch (...) {
    return fail(c, BBC_ENOMEM, "host allocation failed");
  }
  for (int r = 0; r <= p.n_out; r++) row_ptr[r] = p.row_ptr[r];
  for (size_t t = 0; t < p.tasks.size(); t++) {
    const bbc::PairTask& k = p.tasks[t];
    int* o = tasks + 24 * t;
    o[0] = k.nA; o[1] = k.nB; o[2] = k.n1; o[3] = k.n2;
    o[4] = k.sA1; o[5] = k.sA2; o[6] = k.sB1; o[7] = k.sB2;
    for (int i = 0; i < 8; i++) { o[8 + i] = i < k.nA ? k.offA[i] : 0; o[16 + i] = i < k.nB ? k.offB[i] : 0; }
  }
  for (size_t i = 0; i < p.tcontrib_ptr.size(); i++) out_ptr[i] = p.tcontrib_ptr[i];
  for (size_t i = 0; i < p.tcontrib_item.size(); i++) { items[i] = p.tcontrib_item[i]; coefs[i] = p.tcontrib_coef[i]; }
  return BBC_OK;
}

bbc_status bbc_enable_stage_timing(bbc_ctx* c, int enable) {
  if (!c) return BBC_EINVAL;
  cudaError_t e = cudaStreamSynchronize(c->stream);
  if (e != cudaSuccess) return cuda_fail(c, e, "stage timing");
  for (auto& v : c->pending) {
    for (auto& p : v) { c->pool.push_back(p.first); c->pool.push_back(p.second); }
    v.clear();
  }
  c->timing = enable != 0;
  return BBC_OK;
}

bbc_status bbc_stage_timing(bbc_ctx* c, double* ms, long long* launches) {
  if (!c || !ms || !launches) return BBC_EINVAL;
  cudaError_t e = cudaStreamSynchronize(c->stream);
  if (e != cudaSuccess) return cuda_fail(c, e, "stage timing");
  for (int s = 0; s < BBC_N_STAGES; s++) {
    double sum = 0.0;
    for (auto& p : c->pending[s]) {
      float t = 0.f;
      e = cudaEventElapsedTime(&t, p.first, p.second);
      if (e != cudaSuccess) return cuda_fail(c, e, "event time");
      sum += t;
      c->pool.push_back(p.first);
      c->pool.push_back(p.second);
    }
    ms[s] = sum;
    launches[s] = (long long)c->pending[s].size();
    c->pending[s].clear();
  }
  return BBC_OK;
}

bbc_status bbc_launch_counts(const bbc_ctx* c, int* per_load, int* per_build, int* per_contract) {
  if (!c) return BBC_EINVAL;
  // forward and inverse FFT passes: the fused (q-major) layout fuses the x and
  // y passes for L <= 32 (and runs the forward transform as one queue-driven
  // launch there); the field-major layout runs three
  const bool xy = c->fused && c->lat.L <= 32;
  const int passes = xy ? 2 : 3;
  const int fwd = queue_fft(c) ? 1 : passes;
  if (per_load) *per_load = 2;  // absmax, convert
  if (per_build) *per_build = 1 + fwd + (c->prec == BBC_MIXED_BF16 ? 1 : 0);  // build, FFT (, bfloat16 rounding)
  // contraction kernel(s), scales, inverse passes
  if (per_contract) *per_contract = (c->tc ? 2 : c->fused ? 1 : 2) + 1 + passes;
  return BBC_OK;
}

const char* bbc_last_error(const bbc_ctx* c) { return c ? c->err.c_str() : g_create_error.c_str(); }

void bbc_destroy(bbc_ctx* c) { delete c; }

}  // extern "C"
