"""Thin Python binding of libbbc (include/bbc.h): argument marshalling only.

Every function named ``bbc_*`` wraps the C entry point of the same name and
raises :class:`BBCError` on a non-zero status.  :class:`Correlators` strings
the calls together for whole time-slice ranges, using PyTorch only for
device memory (the workspace and outputs) and the CUDA stream.

There is no fallback: if ``libbbc.so`` has not been built the import fails.
"""
from __future__ import annotations

import ctypes
import os

PKG = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(PKG, "libbbc.so")

BBC_OK, BBC_EINVAL, BBC_ENOMEM, BBC_ECUDA, BBC_ESTATE, BBC_ETIMEOUT, BBC_ENUMERIC = 0, -1, -2, -3, -4, -5, -6
BBC_FP64, BBC_MIXED_FP32, BBC_MIXED_BF16, BBC_DF64, BBC_MIXED_TF32 = 0, 1, 2, 3, 4
BBC_UPPER, BBC_LOWER = 0, 1
BBC_C128, BBC_C64 = 0, 1
BBC_LIGHT, BBC_STRANGE = 0, 1

STATUS_NAMES = {0: "OK", -1: "EINVAL", -2: "ENOMEM", -3: "ECUDA", -4: "ESTATE", -5: "ETIMEOUT", -6: "ENUMERIC"}

#: the 52 channels of Sec. 4 in printed order (ids 52..55: the 4 omitted
#: ones, 56..63: other charge states)
CHANNELS_52 = list(range(52))
#: decuplet channels (Sec. 4 footnote, Gamma1 = C gamma_l): Omega Omega and
#: p Omega; Delta++ Delta++, Sigma*+ Sigma*+, Xi*0 Xi*0 (81 vector combinations
#: each) and p Delta++
OMEGA_OMEGA = list(range(64, 145))
P_OMEGA = list(range(145, 154))
DELTA_DELTA = list(range(154, 235))
SIGMA_STAR_PAIRS = list(range(235, 316))
XI_STAR_PAIRS = list(range(316, 397))
P_DELTA = list(range(397, 406))
N_CHANNEL_IDS = 406
DECUPLET_PAIR_BASE = {"Omega": 64, "Delta++": 154, "Sigma*+": 235, "Xi*0": 316}


def omega_channel(l1: int, l2: int, l3: int, l4: int) -> int:
    """Id of Omega_l1 Omega_l2 <- Omega_l3 Omega_l4 (l = 0, 1, 2 for x, y, z)."""
    return decuplet_channel("Omega", l1, l2, l3, l4)


def decuplet_channel(family: str, l1: int, l2: int, l3: int, l4: int) -> int:
    """Id of D_l1 D_l2 <- D_l3 D_l4, D one of Omega, Delta++, Sigma*+, Xi*0."""
    if not all(0 <= v < 3 for v in (l1, l2, l3, l4)):
        raise ValueError("vector indices are 0, 1, 2")
    return DECUPLET_PAIR_BASE[family] + 27 * l1 + 9 * l2 + 3 * l3 + l4


def p_delta_channel(l: int, lp: int) -> int:
    """Id of p Delta++_l <- p Delta++_l'."""
    if not (0 <= l < 3 and 0 <= lp < 3):
        raise ValueError("vector indices are 0, 1, 2")
    return 397 + 3 * l + lp


def p_omega_channel(l: int, lp: int) -> int:
    """Id of p Omega_l <- p Omega_l'."""
    if not (0 <= l < 3 and 0 <= lp < 3):
        raise ValueError("vector indices are 0, 1, 2")
    return 145 + 3 * l + lp


class BBCError(RuntimeError):
    def __init__(self, status: int, message: str):
        super().__init__(f"{STATUS_NAMES.get(status, status)}: {message}")
        self.status = status


class bbc_tuning(ctypes.Structure):
    _fields_ = [("build_sites", ctypes.c_int), ("build_threads", ctypes.c_int),
                ("fused_warps", ctypes.c_int), ("fused_chunk", ctypes.c_int), ("fused_steps", ctypes.c_int),
                ("pair_groups", ctypes.c_int), ("tc_kernel", ctypes.c_int)]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_}


class bbc_batch_item(ctypes.Structure):
    _fields_ = [("ctx", ctypes.c_void_p), ("t", ctypes.c_int), ("S_light", ctypes.c_void_p),
                ("S_strange", ctypes.c_void_p), ("dtype", ctypes.c_int), ("on_device", ctypes.c_int),
                ("out_dev", ctypes.c_void_p), ("normalised", ctypes.c_int)]


class bbc_lattice(ctypes.Structure):
    _fields_ = [("L", ctypes.c_int), ("T", ctypes.c_int), ("t0", ctypes.c_int),
                ("m_ud", ctypes.c_double), ("m_s", ctypes.c_double)]


def _load():
    if not os.path.exists(LIB_PATH):
        raise ImportError(f"libbbc.so not built ({LIB_PATH}); run paper_1510_00903_gb300.build.build()")
    lib = ctypes.CDLL(LIB_PATH)
    P, I, LL = ctypes.c_void_p, ctypes.c_int, ctypes.c_longlong
    sig = {
        "bbc_create": ([ctypes.POINTER(P), ctypes.POINTER(bbc_lattice), I, ctypes.POINTER(I), I, P], I),
        "bbc_create_components": ([ctypes.POINTER(P), ctypes.POINTER(bbc_lattice), I, ctypes.POINTER(I), I, I, P], I),
        "bbc_workspace_size": ([P, I, ctypes.POINTER(ctypes.c_size_t)], I),
        "bbc_set_workspace": ([P, P, ctypes.c_size_t, I], I),
        "bbc_load_propagator": ([P, I, I, I, P, I, I], I),
        "bbc_build_blocks": ([P, I], I),
        "bbc_contract": ([P, I, P, I], I),
        "bbc_plan_stats": ([P, I, I, I, ctypes.POINTER(I), ctypes.POINTER(I), I], I),
        "bbc_plan_sizes": ([P, ctypes.POINTER(I), ctypes.POINTER(I), ctypes.POINTER(I), ctypes.POINTER(LL)], I),
        "bbc_plan_export": ([P, P, P, P, P, P, P, P], I),
        "bbc_enable_stage_timing": ([P, I], I),
        "bbc_stage_timing": ([P, ctypes.POINTER(ctypes.c_double), ctypes.POINTER(LL)], I),
        "bbc_launch_counts": ([P, ctypes.POINTER(I), ctypes.POINTER(I), ctypes.POINTER(I)], I),
        "bbc_run_slice_static": ([P, I, P, P, I, P, I], I),
        "bbc_project": ([P, P, I, P, P], I),
        "bbc_set_checks": ([P, I], I),
        "bbc_device_status": ([P], I),
        "bbc_check_bounded_wait": ([P, LL], I),
        "bbc_batch_run": ([ctypes.POINTER(bbc_batch_item), I, P, ctypes.POINTER(I)], I),
        "bbc_get_tuning": ([P, ctypes.POINTER(bbc_tuning)], I),
        "bbc_set_tuning": ([P, ctypes.POINTER(bbc_tuning)], I),
        "bbc_autotune": ([P, I, ctypes.POINTER(bbc_tuning), ctypes.POINTER(ctypes.c_double), I,
                          ctypes.POINTER(I)], I),
        "bbc_last_error": ([P], ctypes.c_char_p),
        "bbc_destroy": ([P], None),
    }
    for name, (args, res) in sig.items():
        f = getattr(lib, name)
        f.argtypes = args
        f.restype = res
    return lib


_lib = _load()


def lib():
    return _lib


def _check(ctx, status: int):
    if status != BBC_OK:
        msg = _lib.bbc_last_error(ctx)
        raise BBCError(status, msg.decode() if msg else "")


# ----------------------------------------------------------- C entry points
def bbc_create(L: int, T: int, t0: int, m_ud: float, m_s: float, precision: int, channels,
               cuda_stream: int = 0):
    lat = bbc_lattice(L, T, t0, m_ud, m_s)
    ch = (ctypes.c_int * len(channels))(*[int(c) for c in channels])
    ctx = ctypes.c_void_p()
    st = _lib.bbc_create(ctypes.byref(ctx), ctypes.byref(lat), int(precision), ch, len(channels),
                         ctypes.c_void_p(cuda_stream or None))
    _check(None, st)
    return ctx


def bbc_create_components(L: int, T: int, t0: int, m_ud: float, m_s: float, precision: int, channels,
                          components: int, cuda_stream: int = 0):
    lat = bbc_lattice(L, T, t0, m_ud, m_s)
    ch = (ctypes.c_int * len(channels))(*[int(c) for c in channels])
    ctx = ctypes.c_void_p()
    st = _lib.bbc_create_components(ctypes.byref(ctx), ctypes.byref(lat), int(precision), ch, len(channels),
                                    int(components), ctypes.c_void_p(cuda_stream or None))
    _check(None, st)
    return ctx


def bbc_workspace_size(ctx, slices: int) -> int:
    n = ctypes.c_size_t()
    _check(ctx, _lib.bbc_workspace_size(ctx, slices, ctypes.byref(n)))
    return n.value


def bbc_set_workspace(ctx, dev_ptr: int, nbytes: int, slices: int):
    _check(ctx, _lib.bbc_set_workspace(ctx, ctypes.c_void_p(dev_ptr), nbytes, slices))


def bbc_load_propagator(ctx, flavour: int, slot: int, t: int, ptr: int, dtype: int, on_device: bool):
    _check(ctx, _lib.bbc_load_propagator(ctx, flavour, slot, t, ctypes.c_void_p(ptr), dtype, int(on_device)))


def bbc_build_blocks(ctx, n_slots: int):
    _check(ctx, _lib.bbc_build_blocks(ctx, n_slots))


def bbc_contract(ctx, slot: int, out_ptr: int, normalised: bool):
    _check(ctx, _lib.bbc_contract(ctx, slot, ctypes.c_void_p(out_ptr), int(normalised)))


def bbc_plan_stats(ctx, channel_pos: int, term3: int, term4: int, cap: int = 64):
    n = ctypes.c_int()
    buf = (ctypes.c_int * cap)()
    _check(ctx, _lib.bbc_plan_stats(ctx, channel_pos, term3, term4, ctypes.byref(n), buf, cap))
    return [buf[i] for i in range(min(n.value, cap))]


def bbc_plan_sizes(ctx):
    a, b, c, d = ctypes.c_int(), ctypes.c_int(), ctypes.c_int(), ctypes.c_longlong()
    _check(ctx, _lib.bbc_plan_sizes(ctx, ctypes.byref(a), ctypes.byref(b), ctypes.byref(c), ctypes.byref(d)))
    return {"blocks": a.value, "block_outputs": b.value, "pair_items": c.value, "pair_macs_per_site": d.value}


def bbc_plan_export(ctx) -> dict:
    """The plan's host tables (see include/bbc.h): block rows as weighted sums
    of sink-tensor entries, the block-pair tasks and the signed sums."""
    import numpy as np
    sizes = np.zeros(5, dtype=np.int32)
    _check(ctx, _lib.bbc_plan_export(ctx, sizes.ctypes.data, None, None, None, None, None, None))
    n_out, n_terms, n_tasks, n_items, n_outputs = (int(x) for x in sizes)  # also the capacities below
    t = {"row_ptr": np.zeros(n_out + 1, np.int32), "terms": np.zeros((n_terms, 3), np.int32),
         "tasks": np.zeros((n_tasks, 24), np.int32), "out_ptr": np.zeros(n_outputs + 1, np.int32),
         "items": np.zeros(n_items, np.int32), "coefs": np.zeros(n_items, np.float64)}
    _check(ctx, _lib.bbc_plan_export(ctx, sizes.ctypes.data, *(t[k].ctypes.data for k in
                                                               ("row_ptr", "terms", "tasks", "out_ptr", "items",
                                                                "coefs"))))
    return t


def tuning_cache_key(device_name: str, L: int, precision: int, components: int, channels) -> str:
    """Key of a tuned launch configuration: it depends on the GPU model and on
    the problem (lattice extent, precision, spin components, channel list)."""
    return f"{device_name}|L={L}|prec={precision}|comp={components}|ch={','.join(str(int(c)) for c in channels)}"


def tuning_cache_load(path: str) -> dict:
    """{key: configuration} from a cache file ({} if it does not exist or is not valid JSON)."""
    import json
    try:
        with open(path) as f:
            data = json.load(f)
    except (OSError, ValueError):
        return {}
    return data if isinstance(data, dict) else {}


def tuning_cache_store(path: str, key: str, cfg: dict):
    """Add one configuration to a cache file (written to a temporary file,
    then renamed over the old one, so a reader never sees half a file)."""
    import json
    data = tuning_cache_load(path)
    data[key] = {k: int(v) for k, v in cfg.items()}
    tmp = f"{path}.tmp{os.getpid()}"
    with open(tmp, "w") as f:
        json.dump(data, f, indent=1, sort_keys=True)
    os.replace(tmp, path)


STAGES = ["ingest", "build", "fft_fwd", "contract", "fft_inv", "normalise", "wick", "project"]


def bbc_enable_stage_timing(ctx, enable: bool):
    _check(ctx, _lib.bbc_enable_stage_timing(ctx, int(enable)))


def bbc_stage_timing(ctx):
    """{stage: (summed ms, launches)} since timing was enabled or last read."""
    ms = (ctypes.c_double * len(STAGES))()
    n = (ctypes.c_longlong * len(STAGES))()
    _check(ctx, _lib.bbc_stage_timing(ctx, ms, n))
    return {s: (ms[i], n[i]) for i, s in enumerate(STAGES)}


def bbc_launch_counts(ctx):
    a, b, c = ctypes.c_int(), ctypes.c_int(), ctypes.c_int()
    _check(ctx, _lib.bbc_launch_counts(ctx, ctypes.byref(a), ctypes.byref(b), ctypes.byref(c)))
    return {"load": a.value, "build": b.value, "contract": c.value}


def bbc_run_slice_static(ctx, t: int, light_ptr: int, strange_ptr: int, dtype: int, out_ptr: int,
                         normalised: bool):
    """One slice with all device scratch in the library's static array (no
    device allocation); see include/bbc.h for the size limit and sharing."""
    _check(ctx, _lib.bbc_run_slice_static(ctx, t, ctypes.c_void_p(light_ptr), ctypes.c_void_p(strange_ptr), dtype,
                                          ctypes.c_void_p(out_ptr), int(normalised)))


def bbc_project(ctx, c_ptr: int, n_fields: int, r_ptr, ra1_ptr):
    """Source spin states |J M> (R) and their cubic-group A1 average (Ra1) of
    correlators [n_fields][L^3][16]; either output pointer may be None."""
    _check(ctx, _lib.bbc_project(ctx, ctypes.c_void_p(c_ptr), n_fields,
                                 ctypes.c_void_p(r_ptr) if r_ptr else None,
                                 ctypes.c_void_p(ra1_ptr) if ra1_ptr else None))


def bbc_batch_run(items, n_items: int, cuda_stream: int = 0):
    """Run a ctypes array of bbc_batch_item in order on one stream."""
    failed = ctypes.c_int(-1)
    st = _lib.bbc_batch_run(items, n_items, ctypes.c_void_p(cuda_stream or None), ctypes.byref(failed))
    if st != BBC_OK:
        ctx = items[failed.value].ctx if 0 <= failed.value < n_items else None
        msg = _lib.bbc_last_error(ctx)
        raise BBCError(st, f"batch item {failed.value}: " + (msg.decode() if msg else ""))


BBC_CHECK_INPUT, BBC_CHECK_OUTPUT = 1, 2


def bbc_set_checks(ctx, flags: int):
    """Enable numeric checks: BBC_CHECK_INPUT | BBC_CHECK_OUTPUT (ENUMERIC on NaN/inf)."""
    _check(ctx, _lib.bbc_set_checks(ctx, int(flags)))


def bbc_device_status(ctx):
    """Synchronise the context stream; raise BBCError(BBC_ETIMEOUT) if a bounded
    wait of the queue-driven forward FFT gave up since the last call."""
    _check(ctx, _lib.bbc_device_status(ctx))


def bbc_check_bounded_wait(ctx, spin_limit: int) -> int:
    """Self-test of the bounded waits; returns the status (BBC_ETIMEOUT expected)."""
    return int(_lib.bbc_check_bounded_wait(ctx, int(spin_limit)))


def bbc_get_tuning(ctx) -> dict:
    t = bbc_tuning()
    _check(ctx, _lib.bbc_get_tuning(ctx, ctypes.byref(t)))
    return t.as_dict()


def bbc_set_tuning(ctx, build_sites: int, build_threads: int, fused_warps: int = 16, fused_chunk: int = 18,
                   fused_steps: int = 1, pair_groups: int = 0, tc_kernel: int = -1):
    """pair_groups 0 and tc_kernel -1 keep the context's current values."""
    cur = bbc_get_tuning(ctx)
    if pair_groups == 0:
        pair_groups = cur["pair_groups"]
    if tc_kernel == -1:
        tc_kernel = cur["tc_kernel"]
    t = bbc_tuning(build_sites, build_threads, fused_warps, fused_chunk, fused_steps, pair_groups, tc_kernel)
    _check(ctx, _lib.bbc_set_tuning(ctx, ctypes.byref(t)))


def bbc_autotune(ctx, reps: int = 5):
    """Times every candidate launch configuration on slot 0 and keeps the
    fastest; returns (chosen configuration, [ms per candidate])."""
    t = bbc_tuning()
    ms = (ctypes.c_double * 64)()
    n = ctypes.c_int()
    _check(ctx, _lib.bbc_autotune(ctx, reps, ctypes.byref(t), ms, 64, ctypes.byref(n)))
    return t.as_dict(), [ms[i] for i in range(min(n.value, 64))]


def bbc_last_error(ctx) -> str:
    m = _lib.bbc_last_error(ctx)
    return m.decode() if m else ""


def bbc_destroy(ctx):
    _lib.bbc_destroy(ctx)


# ------------------------------------------------------------ convenience
class Correlators:
    """All steps of the path for one lattice, on one CUDA stream.

    ``run(S_light, S_strange, times)`` takes propagators ``[len(times), V, 12, 12]``
    (torch tensors, complex128 or complex64, on the GPU or pinned on the host)
    and returns ``[len(times), n_channels, V, 16]`` complex128 on the GPU.
    """

    def __init__(self, L: int, T: int, t0: int = 0, m_ud: float = 0.3, m_s: float = 0.4,
                 channels=CHANNELS_52, precision: int = BBC_FP64, slices: int = 1, device=None,
                 stream=None, workspace=None, components: int = BBC_UPPER):
        import torch
        self.torch = torch
        dev = torch.device(device or "cuda")
        if dev.index is None:
            dev = torch.device("cuda", torch.cuda.current_device())
        self.device = dev
        self.stream = stream or torch.cuda.current_stream(self.device)
        self.L, self.T, self.t0, self.V = L, T, t0, L ** 3
        self.channels = list(channels)
        self.precision = precision
        self.components = components
        self.ctx = bbc_create_components(L, T, t0, m_ud, m_s, precision, self.channels, components,
                                         self.stream.cuda_stream)
        self.slices = slices
        nbytes = bbc_workspace_size(self.ctx, slices)
        if workspace is None:
            workspace = torch.empty(nbytes + 256, dtype=torch.uint8, device=self.device)
        elif workspace.numel() < nbytes + 256:
            raise ValueError(f"workspace needs {nbytes + 256} bytes")
        # contexts whose work is ordered on one stream may share a workspace
        self.workspace = workspace
        base = self.workspace.data_ptr()
        self._ws_ptr = (base + 255) // 256 * 256
        with torch.cuda.stream(self.stream):
            bbc_set_workspace(self.ctx, self._ws_ptr, nbytes, slices)

    def sizes(self):
        return bbc_plan_sizes(self.ctx)

    def load(self, flavour: int, slot: int, t: int, S):
        torch = self.torch
        dtype = {torch.complex128: BBC_C128, torch.complex64: BBC_C64}[S.dtype]
        if not S.is_contiguous() or S.numel() != self.V * 144:
            raise ValueError(f"propagator slice must be contiguous [{self.V}, 12, 12]")
        if S.is_cuda and S.device != self.device:
            raise ValueError("propagator on another device")
        bbc_load_propagator(self.ctx, flavour, slot, t, S.data_ptr(), dtype, S.is_cuda)

    def build(self, n_slots: int):
        bbc_build_blocks(self.ctx, n_slots)

    def contract(self, slot: int, out, normalised: bool = True):
        if out.dtype != self.torch.complex128 or not out.is_cuda or not out.is_contiguous():
            raise ValueError("out must be a contiguous complex128 CUDA tensor")
        bbc_contract(self.ctx, slot, out.data_ptr(), normalised)

    def run(self, S_light, S_strange, times, out=None, normalised: bool = True):
        torch = self.torch
        times = list(times)
        n_ch = len(self.channels)
        if out is None:
            out = torch.empty((len(times), n_ch, self.V, 16), dtype=torch.complex128, device=self.device)
        # inputs and output were written or allocated on the caller's stream
        cur = torch.cuda.current_stream(self.device)
        if cur.cuda_stream != self.stream.cuda_stream:
            self.stream.wait_stream(cur)
        with torch.cuda.stream(self.stream):
            for i0 in range(0, len(times), self.slices):
                chunk = times[i0:i0 + self.slices]
                for j, t in enumerate(chunk):
                    self.load(BBC_LIGHT, j, t, S_light[i0 + j])
                    self.load(BBC_STRANGE, j, t, S_strange[i0 + j])
                self.build(len(chunk))
                for j in range(len(chunk)):
                    self.contract(j, out[i0 + j], normalised)
        # the caller's stream sees the results (and may free the inputs) only
        # after the work queued on the context stream
        if cur.cuda_stream != self.stream.cuda_stream:
            cur.wait_stream(self.stream)
        return out

    def run_streamed(self, S_light, S_strange, times, out, normalised: bool = True, on_slice=None):
        """Slices whose propagators live in pinned host memory ([T, V, 12, 12]):
        the host-to-device copy of slice i+1 (on a copy stream, into one of
        two device buffers) overlaps the compute of slice i.  The correlators
        of each slice land in ``out`` ([n_channels, V, 16], overwritten slice
        after slice); ``on_slice(t, out)``, if given, is called after each
        slice's work is queued, to queue a consumer on the context stream."""
        torch = self.torch
        times = list(times)
        if not times:
            return out
        V = self.V
        key = (S_light.dtype, S_strange.dtype)
        if getattr(self, "_stream_key", None) != key:
            self._copy_stream = torch.cuda.Stream(self.device)
            self._stream_bufs = [(torch.empty((V, 12, 12), dtype=S_light.dtype, device=self.device),
                                  torch.empty((V, 12, 12), dtype=S_strange.dtype, device=self.device))
                                 for _ in range(2)]
            self._stream_key = key
        copy, bufs = self._copy_stream, self._stream_bufs
        copied = [torch.cuda.Event() for _ in range(2)]
        consumed = [torch.cuda.Event() for _ in range(2)]
        cur = torch.cuda.current_stream(self.device)
        if cur.cuda_stream != self.stream.cuda_stream:
            self.stream.wait_stream(cur)
        copy.wait_stream(self.stream)  # earlier readers of the buffers

        def issue_copy(i):
            b = i % 2
            with torch.cuda.stream(copy):
                if i >= 2:
                    copy.wait_event(consumed[b])
                bufs[b][0].copy_(S_light[times[i]], non_blocking=True)
                bufs[b][1].copy_(S_strange[times[i]], non_blocking=True)
                copied[b].record(copy)

        issue_copy(0)
        for i, t in enumerate(times):
            if i + 1 < len(times):
                issue_copy(i + 1)
            b = i % 2
            with torch.cuda.stream(self.stream):
                self.stream.wait_event(copied[b])
                self.load(BBC_LIGHT, 0, t, bufs[b][0])
                self.load(BBC_STRANGE, 0, t, bufs[b][1])
                consumed[b].record(self.stream)
                self.build(1)
                self.contract(0, out, normalised)
                if on_slice is not None:
                    on_slice(t, out)
        if cur.cuda_stream != self.stream.cuda_stream:
            cur.wait_stream(self.stream)
        return out

    def run_each(self, S_light, S_strange, times, out, normalised: bool = True, on_slice=None):
        """Slices whose propagators are already on the device ([T, V, 12, 12]):
        one slice after the other through the context's first slot, every
        slice's correlators written into the same ``out`` ([n_channels, V,
        16]); ``on_slice(t, out)``, if given, is called after each slice's work
        is queued (to queue a consumer on the context stream)."""
        torch = self.torch
        cur = torch.cuda.current_stream(self.device)
        if cur.cuda_stream != self.stream.cuda_stream:
            self.stream.wait_stream(cur)
        with torch.cuda.stream(self.stream):
            for t in times:
                self.load(BBC_LIGHT, 0, t, S_light[t])
                self.load(BBC_STRANGE, 0, t, S_strange[t])
                self.build(1)
                self.contract(0, out, normalised)
                if on_slice is not None:
                    on_slice(t, out)
        if cur.cuda_stream != self.stream.cuda_stream:
            cur.wait_stream(self.stream)
        return out

    def run_to_host(self, S_light, S_strange, times, out_host, normalised: bool = True):
        """End to end from pinned host propagators ([T, V, 12, 12]) to pinned
        host correlators out_host [len(times), n_channels, V, 16] complex128:
        the host-to-device copy of slice i+1, the compute of slice i and the
        device-to-host copy of slice i-1 overlap (two copy streams, double
        buffers on the device).  An out_host of R < len(times) slices is used
        as a ring: slice i lands in out_host[i % R] (a consumer reads it before
        slice i + R is copied there)."""
        torch = self.torch
        times = list(times)
        if not times:
            return out_host
        n_ch = len(self.channels)
        if getattr(self, "_d2h_bufs", None) is None:
            self._d2h_stream = torch.cuda.Stream(self.device)
            self._d2h_bufs = [torch.empty((n_ch, self.V, 16), dtype=torch.complex128, device=self.device)
                              for _ in range(2)]
        d2h, obufs = self._d2h_stream, self._d2h_bufs
        done = [torch.cuda.Event() for _ in range(2)]
        drained = [torch.cuda.Event() for _ in range(2)]
        state = {"i": 0}

        def on_slice(t, out):
            i = state["i"]
            b = i % 2
            if i >= 2:
                self.stream.wait_event(drained[b])  # the copy out of this buffer two slices ago
            # the slice was written into the shared buffer: move it to its own one
            obufs[b].copy_(out, non_blocking=True)
            done[b].record(self.stream)
            with torch.cuda.stream(d2h):
                d2h.wait_event(done[b])
                out_host[i % out_host.shape[0]].copy_(obufs[b], non_blocking=True)
                drained[b].record(d2h)
            state["i"] = i + 1

        out = self._d2h_out = getattr(self, "_d2h_out", None)
        if out is None:
            out = self._d2h_out = torch.empty((n_ch, self.V, 16), dtype=torch.complex128, device=self.device)
        d2h.wait_stream(self.stream)
        self.run_streamed(S_light, S_strange, times, out, normalised, on_slice=on_slice)
        cur = torch.cuda.current_stream(self.device)
        cur.wait_stream(d2h)
        if cur.cuda_stream != self.stream.cuda_stream:
            cur.wait_stream(self.stream)
        return out_host

    def autotune(self, S_light, S_strange, t: int = 0, reps: int = 5, cache: str | None = None):
        """Load slice t into slot 0 and run the autotuner (bbc_autotune);
        returns (configuration, ms per candidate).

        cache: a JSON file of tuned configurations (default: the
        BBC_AUTOTUNE_CACHE environment variable, if set).  A configuration
        stored there for this GPU model, L, precision, spin components and
        channel list is applied without timing (ms is then empty); otherwise
        the tuned one is added to it."""
        torch = self.torch
        path = cache if cache is not None else os.environ.get("BBC_AUTOTUNE_CACHE")
        key = None
        if path:
            key = tuning_cache_key(torch.cuda.get_device_name(self.device), self.L, self.precision,
                                   self.components, self.channels)
            cached = tuning_cache_load(path).get(key)
            if cached is not None:
                self.set_tuning(cached)
                return self.tuning(), []
        cur = torch.cuda.current_stream(self.device)
        if cur.cuda_stream != self.stream.cuda_stream:
            self.stream.wait_stream(cur)
        with torch.cuda.stream(self.stream):
            self.load(BBC_LIGHT, 0, t, S_light)
            self.load(BBC_STRANGE, 0, t, S_strange)
            cfg, ms = bbc_autotune(self.ctx, reps)
        if path:
            tuning_cache_store(path, key, cfg)
        return cfg, ms

    def status(self):
        """Synchronise and raise BBCError(BBC_ETIMEOUT) if a bounded device wait gave up."""
        bbc_device_status(self.ctx)

    def tuning(self) -> dict:
        return bbc_get_tuning(self.ctx)

    def set_tuning(self, cfg: dict):
        bbc_set_tuning(self.ctx, cfg["build_sites"], cfg["build_threads"], cfg["fused_warps"], cfg["fused_chunk"],
                       cfg.get("fused_steps", 1), cfg.get("pair_groups", 0), cfg.get("tc_kernel", -1))

    def project(self, C, R=None, Ra1=None, a1: bool = True):
        """Spin states |J M> and, with ``a1``, the cubic-group A1 average of
        correlators C [..., V, 16] complex128 on the GPU (bbc_project).
        Returns (R, Ra1); Ra1 is None without ``a1``."""
        torch = self.torch
        if C.dtype != torch.complex128 or not C.is_cuda or not C.is_contiguous() or C.shape[-2:] != (self.V, 16):
            raise ValueError(f"C must be a contiguous complex128 CUDA tensor [..., {self.V}, 16]")
        n_fields = C.numel() // (self.V * 16)
        if R is None:
            R = torch.empty_like(C)
        if a1 and Ra1 is None:
            Ra1 = torch.empty_like(C)
        cur = torch.cuda.current_stream(self.device)
        if cur.cuda_stream != self.stream.cuda_stream:
            self.stream.wait_stream(cur)
        with torch.cuda.stream(self.stream):
            bbc_project(self.ctx, C.data_ptr(), n_fields, R.data_ptr(), Ra1.data_ptr() if a1 else None)
        if cur.cuda_stream != self.stream.cuda_stream:
            cur.wait_stream(self.stream)
        return R, (Ra1 if a1 else None)

    def capture(self, S_light, S_strange, times, out, normalised: bool = True):
        """Record run(...) for these slices into one CUDA graph (after an eager
        run that sets kernel attributes); replaying the graph repeats the
        whole computation into `out` with one launch.  Needs a non-default
        stream (pass `stream=torch.cuda.Stream()` at construction)."""
        torch = self.torch
        if self.stream.cuda_stream == 0:
            raise ValueError("graph capture needs a non-default stream")
        self.run(S_light, S_strange, times, out=out, normalised=normalised)
        torch.cuda.synchronize(self.device)
        g = torch.cuda.CUDAGraph()
        with torch.cuda.graph(g, stream=self.stream):
            self.run(S_light, S_strange, times, out=out, normalised=normalised)
        return g

    def close(self):
        if self.ctx:
            bbc_destroy(self.ctx)
            self.ctx = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class LatticeBatch:
    """Several lattices and wall sources run as one CUDA graph on one stream.

    ``lattices``: list of (L, T); every lattice runs ``n_sources`` wall
    sources at t0 = 0, T/n, 2T/n, ...  Contexts of one lattice share one
    workspace (their work is ordered on the stream).  ``inputs[i]`` =
    (S_light, S_strange), each [T, V, 12, 12] on the device, serve every source
    of lattice i.  ``run()`` computes every slice of every source; the
    correlators of a slice land in ``outputs[i]`` ([n_channels, V, 16]),
    overwritten slice after slice (a streaming consumer reads them there).
    Each context holds ``slices`` slots: bbc_batch_run takes a source's slices
    in waves of that many (one block build and one forward FFT per wave).
    """

    def __init__(self, lattices, inputs, n_sources: int = 4, channels=CHANNELS_52,
                 precision: int = BBC_MIXED_FP32, m_ud: float = 0.3, m_s: float = 0.4, device=None,
                 slices: int = 4):
        import torch
        self.torch = torch
        dev = torch.device(device or "cuda")
        if dev.index is None:
            dev = torch.device("cuda", torch.cuda.current_device())
        self.device = dev
        self.stream = torch.cuda.Stream(dev)
        self.lattices, self.inputs, self.n_sources = list(lattices), list(inputs), n_sources
        self.cors, self.outputs = [], []
        for (L, T), _ in zip(self.lattices, self.inputs):
            per = []
            ws = None
            for k in range(n_sources):
                c = Correlators(L, T, (k * T) // n_sources, m_ud, m_s, channels=channels, precision=precision,
                                slices=min(slices, T), device=dev, stream=self.stream, workspace=ws)
                ws = c.workspace
                per.append(c)
            self.cors.append(per)
            self.outputs.append(torch.empty((len(channels), L ** 3, 16), dtype=torch.complex128, device=dev))
        # one batch item per (lattice, source, slice), in that order
        n = sum(len(per) * per[0].T for per in self.cors)
        self._items = (bbc_batch_item * n)()
        i = 0
        for per, (Sl, Ss), out in zip(self.cors, self.inputs, self.outputs):
            dt = {torch.complex128: BBC_C128, torch.complex64: BBC_C64}[Sl.dtype]
            if Ss.dtype != Sl.dtype or not (Sl.is_cuda and Ss.is_cuda and Sl.is_contiguous() and Ss.is_contiguous()):
                raise ValueError("inputs must be contiguous CUDA tensors of one dtype")
            for c in per:
                for t in range(c.T):
                    self._items[i] = bbc_batch_item(c.ctx, t, Sl[t].data_ptr(), Ss[t].data_ptr(), dt, 1,
                                                    out.data_ptr(), 1)
                    i += 1
        self._n_items = n

    def sites_channels(self) -> int:
        n_ch = self.outputs[0].shape[0]
        return sum(self.n_sources * T * L ** 3 * n_ch for (L, T) in self.lattices)

    def run(self):
        torch = self.torch
        cur = torch.cuda.current_stream(self.device)
        if cur.cuda_stream != self.stream.cuda_stream:
            self.stream.wait_stream(cur)
        with torch.cuda.stream(self.stream):
            bbc_batch_run(self._items, self._n_items, self.stream.cuda_stream)
        if cur.cuda_stream != self.stream.cuda_stream:
            cur.wait_stream(self.stream)

    def autotune(self, reps: int = 3) -> dict:
        """Autotune the first context of every distinct L on its slice 0 and
        give the chosen configuration to every context of that L (before
        capture).  Returns {L: configuration}."""
        chosen = {}
        for per, (Sl, Ss) in zip(self.cors, self.inputs):
            L = per[0].L
            if L not in chosen:
                chosen[L], _ = per[0].autotune(Sl[0], Ss[0], t=0, reps=reps)
            for c in per:
                c.set_tuning(chosen[L])
        return chosen

    def capture(self):
        """One CUDA graph for every slice of every source of every lattice."""
        torch = self.torch
        self.run()
        torch.cuda.synchronize(self.device)
        g = torch.cuda.CUDAGraph()
        with torch.cuda.graph(g, stream=self.stream):
            self.run()
        return g

    def status(self):
        """Synchronise and raise BBCError(BBC_ETIMEOUT) if a bounded device wait of
        any context gave up."""
        for per in self.cors:
            for c in per:
                c.status()

    def close(self):
        for per in self.cors:
            for c in per:
                c.close()
