// static_scratch.cu -- bbc_run_slice_static: the one entry point of libbbc
// that allocates nothing.
//
// Some callers cannot call cudaMalloc (or ask PyTorch for memory): a host
// program whose device memory is owned by another runtime's pool allocator,
// a plugin loaded into such a process, or a loop that must not hit the
// implicit device synchronisation and failure modes of an allocation.  For
// them this entry point runs one time slice of the whole path (ingest, block
// build, forward FFT, pair products, Wick sums, inverse FFT, normalisation)
// with every byte of device scratch inside one file-scope __device__ array of
// BBC_STATIC_SCRATCH_BYTES.  The array exists on every GPU that loads the
// library, from module load until process exit.  The caller still passes the
// propagators and the output buffer (device pointers).
#include <cmath>
#include <cstring>
#include <mutex>

#include "ctx_internal.hpp"

namespace {

constexpr size_t kStaticScratchBytes = (size_t)BBC_STATIC_SCRATCH_BYTES;
constexpr int kMaxDevices = 64;

// The scratch itself.  Host code must not use this symbol as an address: it
// is a host-side stand-in for the device array; the device address comes from
// cudaGetSymbolAddress below.
static __device__ __align__(256) unsigned char g_static_scratch[kStaticScratchBytes];

std::mutex g_setup_mutex;
void* g_scratch_addr[kMaxDevices] = {nullptr};

size_t a256(size_t x) { return (x + 255) & ~size_t(255); }

struct StaticLayout {
  size_t ell_chunk, ell, zneed, tasks, group_ptr, group_task, cptr, citem, ccoef;
  size_t prop, amax, kexp, blk, blkf, P, ct, scale, total;
};

StaticLayout static_layout(const bbc_ctx* c) {
  const bbc::Plan& p = c->plan;
  const size_t cb = c->prec == BBC_FP64 ? 16 : 8, V = (size_t)c->V;
  StaticLayout L{};
  size_t o = 0;
  L.ell_chunk = o; o = a256(o + sizeof(int2) * p.ell_chunk.size());
  L.ell = o; o = a256(o + sizeof(uint32_t) * p.ell.size());
  L.zneed = o; o = a256(o + sizeof(uint32_t) * p.zneed.size());
  L.tasks = o; o = a256(o + sizeof(bbc::DevTask) * p.tasks.size());
  L.group_ptr = o; o = a256(o + sizeof(int) * c->group_ptr.size());
  L.group_task = o; o = a256(o + sizeof(int) * c->group_task.size());
  L.cptr = o; o = a256(o + sizeof(int) * p.tcontrib_ptr.size());
  L.citem = o; o = a256(o + sizeof(int) * p.tcontrib_item.size());
  L.ccoef = o; o = a256(o + sizeof(double) * p.tcontrib_coef.size());
  L.prop = o; o = a256(o + 2 * V * 144 * cb);
  L.amax = o; o = a256(o + 2 * sizeof(unsigned long long));
  L.kexp = o; o = a256(o + 2 * sizeof(int));
  L.blk = o; o = a256(o + V * p.n_out * cb);
  L.blkf = o; o = a256(o + V * p.n_out * cb);
  L.P = o; o = a256(o + p.tasks.size() * 16 * V * cb);
  L.ct = o; o = a256(o + p.channels.size() * 16 * V * 16);
  L.scale = o; o = a256(o + sizeof(double) * bbc::kMaxChannels);
  L.total = o;
  return L;
}

bbc_status fail(bbc_ctx* c, bbc_status s, const char* msg) {
  c->err = msg;
  return s;
}

bbc_status cuda_fail(bbc_ctx* c, cudaError_t e, const char* where) {
  c->err = std::string(where) + ": " + cudaGetErrorString(e);
  return BBC_ECUDA;
}

}  // namespace

extern "C" bbc_status bbc_run_slice_static(bbc_ctx* c, int t, const void* S_light, const void* S_strange,
                                           int dtype, void* out_dev, int normalised) {
  if (!c) return BBC_EINVAL;
  if (t < 0 || t >= c->lat.T) return fail(c, BBC_EINVAL, "bad time slice");
  if (dtype != BBC_C128 && dtype != BBC_C64) return fail(c, BBC_EINVAL, "bad dtype");
  if (c->prec != BBC_FP64 && c->prec != BBC_MIXED_FP32)
    return fail(c, BBC_EINVAL, "the static entry point runs BBC_FP64 and BBC_MIXED_FP32");
  if (c->checks)  // the numeric checks need a flag word and a synchronising read-back
    return fail(c, BBC_EINVAL, "the static entry point runs without numeric checks (bbc_set_checks(ctx, 0))");
  if (!S_light || !S_strange || !out_dev || (((uintptr_t)S_light | (uintptr_t)S_strange | (uintptr_t)out_dev) & 15))
    return fail(c, BBC_EINVAL, "propagators and output must be 16-byte aligned device pointers");
  const StaticLayout L = static_layout(c);
  if (L.total > kStaticScratchBytes)
    return fail(c, BBC_EINVAL,
                "lattice and channel list need more device scratch than the static array holds "
                "(BBC_STATIC_SCRATCH_BYTES = 32 MiB: L <= 4 with all 52 channels)");
  static_assert(BBC_STATIC_SCRATCH_BYTES % 256 == 0, "scratch size");
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return cuda_fail(c, e, "cudaGetDevice");
  if (dev < 0 || dev >= kMaxDevices) return fail(c, BBC_EINVAL, "device index beyond the supported 64");
  char* w;
  {
    // set-up, once per device, with that device current
    std::lock_guard<std::mutex> lock(g_setup_mutex);
    if (!g_scratch_addr[dev]) {
      void* p = nullptr;
      e = cudaGetSymbolAddress(&p, g_static_scratch);
      if (e != cudaSuccess) return cuda_fail(c, e, "cudaGetSymbolAddress(static scratch)");
      g_scratch_addr[dev] = p;
    }
    w = (char*)g_scratch_addr[dev];
  }
  if (!c->twiddles) {
    e = bbc::upload_twiddles();
    if (e != cudaSuccess) return cuda_fail(c, e, "twiddle upload");
    c->twiddles = true;
  }
  const bbc::Plan& p = c->plan;
  cudaStream_t st = c->stream;
  // plan tables (copies from pageable host memory return once the data is staged)
  struct Up { size_t off; const void* src; size_t n; } ups[] = {
      {L.ell_chunk, p.ell_chunk.data(), sizeof(int2) * p.ell_chunk.size()},
      {L.ell, p.ell.data(), sizeof(uint32_t) * p.ell.size()},
      {L.zneed, p.zneed.data(), sizeof(uint32_t) * p.zneed.size()},
      {L.group_ptr, c->group_ptr.data(), sizeof(int) * c->group_ptr.size()},
      {L.group_task, c->group_task.data(), sizeof(int) * c->group_task.size()},
      {L.cptr, p.tcontrib_ptr.data(), sizeof(int) * p.tcontrib_ptr.size()},
      {L.citem, p.tcontrib_item.data(), sizeof(int) * p.tcontrib_item.size()},
      {L.ccoef, p.tcontrib_coef.data(), sizeof(double) * p.tcontrib_coef.size()},
  };
  for (auto& u : ups) {
    if (!u.n) continue;
    e = cudaMemcpyAsync(w + u.off, u.src, u.n, cudaMemcpyHostToDevice, st);
    if (e != cudaSuccess) return cuda_fail(c, e, "table upload");
  }
  // tasks in device format, staged through a fixed stack buffer (no heap use)
  {
    bbc::DevTask buf[64];
    const size_t nt = p.tasks.size();
    for (size_t i0 = 0; i0 < nt; i0 += 64) {
      const size_t n = nt - i0 < 64 ? nt - i0 : 64;
      bbc::to_dev_tasks(p.tasks.data() + i0, n, nullptr, buf);
      e = cudaMemcpyAsync(w + L.tasks + i0 * sizeof(bbc::DevTask), buf, n * sizeof(bbc::DevTask),
                          cudaMemcpyHostToDevice, st);
      if (e != cudaSuccess) return cuda_fail(c, e, "task upload");
    }
  }
  const bool fp64 = c->prec == BBC_FP64;
  const size_t nc = (size_t)c->V * 144, cb = fp64 ? 16 : 8;
  unsigned long long* amax = (unsigned long long*)(w + L.amax);
  int* kexp = (int*)(w + L.kexp);
  // the maxima accumulate with atomicMax: they must start at zero every call
  e = cudaMemsetAsync(amax, 0, 2 * sizeof(unsigned long long), st);
  if (e != cudaSuccess) return cuda_fail(c, e, "memset");
  const void* src[2] = {S_light, S_strange};
  for (int f = 0; f < 2; f++) {
    e = bbc::launch_absmax(src[f], dtype, (long long)nc, amax + f, st);
    if (e != cudaSuccess) return cuda_fail(c, e, "absmax kernel");
    e = bbc::launch_convert(src[f], dtype, (long long)nc, amax + f, kexp + f, w + L.prop + f * nc * cb,
                           fp64 ? bbc::RK_F64 : bbc::RK_F32, st);
    if (e != cudaSuccess) return cuda_fail(c, e, "convert kernel");
  }
  const bbc::DevGroups g = bbc::dev_groups(p);
  e = bbc::launch_block_build(w + L.prop, c->V, 1, (const int2*)(w + L.ell_chunk), (const uint32_t*)(w + L.ell),
                              (const uint32_t*)(w + L.zneed), g, w + L.blk, p.n_out, fp64 ? bbc::RK_F64 : bbc::RK_F32,
                              st, 1, 256);
  if (e != cudaSuccess) return cuda_fail(c, e, "block build");
  e = bbc::launch_fft_forward(w + L.blk, w + L.blkf, c->lat.L, 1, p.n_out, fp64, st);
  if (e != cudaSuccess) return cuda_fail(c, e, "forward FFT");
  e = bbc::launch_pair_products(w + L.blkf, c->lat.L, (const bbc::DevTask*)(w + L.tasks), (const int*)(w + L.group_ptr),
                                (const int*)(w + L.group_task), (int)c->group_ptr.size() - 1, w + L.P, fp64, st);
  if (e != cudaSuccess) return cuda_fail(c, e, "pair products");
  const int n_ch = (int)p.channels.size();
  e = bbc::launch_wick_sums(w + L.P, c->lat.L, (const int*)(w + L.cptr), (const int*)(w + L.citem),
                            (const double*)(w + L.ccoef), n_ch, w + L.ct, fp64, st);
  if (e != cudaSuccess) return cuda_fail(c, e, "Wick sums");
  bbc::ScaleParams sp{};
  sp.n_ch = n_ch;
  const int dt = c->plan.spin_offset ? c->lat.t0 - t : t - c->lat.t0;  // forward or backward in time
  const int d = ((dt % c->lat.T) + c->lat.T) % c->lat.T;
  for (int i = 0; i < n_ch; i++) {
    const int ns = p.n_strange[i];
    const double mass = (6 - ns) * c->lat.m_ud + ns * c->lat.m_s;
    sp.f[i] = (1.0 / c->V) * (normalised ? std::exp(mass * d) : 1.0);
    sp.nl[i] = 6 - ns;
    sp.ns[i] = ns;
  }
  e = bbc::launch_scales(sp, kexp, (double*)(w + L.scale), st);
  if (e != cudaSuccess) return cuda_fail(c, e, "normalisation");
  e = bbc::launch_fft_inverse(w + L.ct, out_dev, c->lat.L, n_ch, (const double*)(w + L.scale), fp64, st);
  if (e != cudaSuccess) return cuda_fail(c, e, "inverse FFT");
  return BBC_OK;
}
