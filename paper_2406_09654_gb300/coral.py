"""Thin Python binding of the C ABI in include/coral.h (ctypes; argument marshalling only).

Every step of the substrate update runs in the CUDA library ``lib/libcoral.so``; this module
only converts arguments. If the library is missing it raises: there is no CPU fallback.
Arrays may be numpy arrays (host memory) or CUDA torch tensors (device memory).
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "lib", "libcoral.so")

OK, E_INVALID, E_OOM, E_CUDA, E_CAPACITY, E_TIMEOUT, E_STATE = 0, -1, -2, -3, -4, -5, -6
FP32_PERCELL, BF16_GROUPED = 0, 1
CH_E, CH_I, CH_C0, CH_C1, CH_C2, CH_C3, CH_G, CH_R = (1 << b for b in range(8))
CH_C = CH_C0 | CH_C1 | CH_C2 | CH_C3
CH_ALL = 0xFF
RING = 4096


class CoralError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__(f"coral error {code}: {msg}")
        self.code = code


class Params(ctypes.Structure):
    _fields_ = [
        ("hidden", ctypes.c_int32), ("path", ctypes.c_int32),
        ("k_inv", ctypes.c_float), ("k_liq", ctypes.c_float), ("k_exp", ctypes.c_float),
        ("k_flow", ctypes.c_float), ("e_day", ctypes.c_float), ("e_night", ctypes.c_float),
        ("day_period", ctypes.c_int32), ("rotation", ctypes.c_int32),
        ("radiation_every", ctypes.c_int32), ("p_mut", ctypes.c_double),
        ("p_merge", ctypes.c_double), ("sigma_mut", ctypes.c_float),
        ("world", ctypes.c_uint32), ("seed", ctypes.c_uint64),
    ]


class Stats(ctypes.Structure):
    _fields_ = [
        ("step", ctypes.c_int64), ("sum_E", ctypes.c_double), ("sum_I", ctypes.c_double),
        ("sum_C", ctypes.c_double * 4), ("n_explore", ctypes.c_int64),
        ("n_takeover", ctypes.c_int64), ("n_live", ctypes.c_int64), ("n_mut", ctypes.c_int64),
        ("n_merge", ctypes.c_int64), ("n_born", ctypes.c_int64), ("n_skipped", ctypes.c_int64),
    ]

    def as_dict(self):
        d = {k: getattr(self, k) for k, _ in self._fields_}
        d["sum_C"] = list(self.sum_C)
        return d


_VP, _I32, _I64, _U32, _SZ = ctypes.c_void_p, ctypes.c_int32, ctypes.c_int64, ctypes.c_uint32, ctypes.c_size_t
STATE_BYTES = 29     # packed state per cell: E, I, C0..C3 float32, G int32, R uint8

SIGNATURES = {
    "coral_params_default": (ctypes.c_int, [ctypes.POINTER(Params)]),
    "coral_substrate_create": (ctypes.c_int, [ctypes.POINTER(Params), _I32, _I32, _I32, _VP,
                                              ctypes.POINTER(_VP)]),
    "coral_substrate_destroy": (ctypes.c_int, [_VP]),
    "coral_state_load": (ctypes.c_int, [_VP, _VP, _VP, _VP, _VP, _VP, ctypes.c_int]),
    "coral_genome_table_load": (ctypes.c_int, [_VP, _I32, _VP, _VP, ctypes.c_int]),
    "coral_cppn_generate_weights": (ctypes.c_int, [_VP, _VP, _I32]),
    "coral_step": (ctypes.c_int, [_VP, _I32]),
    "coral_set_fma_cutoff": (ctypes.c_int, [_VP, _I32]),
    "coral_batch_set_fma_cutoff": (ctypes.c_int, [_VP, _I32]),
    "coral_step_timed": (ctypes.c_int, [_VP, _I32, _VP, _VP]),
    "coral_step_jobs": (ctypes.c_int, [_VP, _I32, _VP, _VP, _I32, _I64]),
    "coral_read_channels": (ctypes.c_int, [_VP, _U32, _VP, _SZ, ctypes.c_int]),
    "coral_read_stats": (ctypes.c_int, [_VP, _I64, _I32, ctypes.POINTER(Stats)]),
    "coral_read_perm": (ctypes.c_int, [_VP, _VP, _VP]),
    "coral_read_genomes": (ctypes.c_int, [_VP, _VP, _VP]),
    "coral_read_weights": (ctypes.c_int, [_VP, _I32, _VP, _SZ]),
    "coral_genome_distances": (ctypes.c_int, [_VP, _VP, _I32, _VP]),
    "coral_set_step": (ctypes.c_int, [_VP, _I64]),
    "coral_get_step": (ctypes.c_int, [_VP, ctypes.POINTER(_I64)]),
    "coral_sync": (ctypes.c_int, [_VP]),
    "coral_launch_config": (ctypes.c_int, [_VP, _VP, _VP, _VP]),
    "coral_selftest_wait_timeout": (ctypes.c_int, [_VP, _I32, _VP]),
    "coral_last_error": (ctypes.c_char_p, [_VP]),
    "coral_net_floats": (_I32, [_I32]),
    "coral_bucket_noalloc": (ctypes.c_int, [_VP, _I64, _I32, _VP, _VP, _VP]),
    "coral_batch_create": (ctypes.c_int, [_VP, _I32, ctypes.POINTER(_VP)]),
    "coral_batch_destroy": (ctypes.c_int, [_VP]),
    "coral_batch_step": (ctypes.c_int, [_VP, _I32]),
    "coral_batch_step_timed": (ctypes.c_int, [_VP, _I32, _VP]),
    "coral_batch_tune": (ctypes.c_int, [_VP, _I32, _VP]),
    "coral_bucket_noalloc_last_error": (ctypes.c_char_p, []),
    "coral_philox4x32_10": (ctypes.c_int, [_VP, _VP, _VP, _I32]),
    "coral_measure_sfu_rate": (ctypes.c_int, [_VP, ctypes.POINTER(ctypes.c_double)]),
    "coral_slab_set": (ctypes.c_int, [_VP, _I32, _I32, _I64]),
    "coral_copy_rows": (ctypes.c_int, [_VP, _I32, _VP, _I32, _I32]),
    "coral_slab_totals": (ctypes.c_int, [_VP, _VP]),
    "coral_slab_radiation_scan": (ctypes.c_int, [_VP, _VP, _VP, _I32, _VP]),
    "coral_slab_radiation_apply": (ctypes.c_int, [_VP, _VP, _VP, _I32, _VP]),
}

_lib = None


def lib():
    """The loaded CUDA library (raises if it was not built)."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise RuntimeError(f"{LIB_PATH} is missing: build it with paper_2406_09654_gb300.build.build()")
        L = ctypes.CDLL(LIB_PATH)
        for name, (res, args) in SIGNATURES.items():
            fn = getattr(L, name)
            fn.restype = res
            fn.argtypes = args
        _lib = L
    return _lib


def _touched(nbytes):
    """A fresh host buffer whose pages the CPU has already faulted in: a device copy into
    untouched pageable memory pays the page faults at a few GB/s, the CPU at memset speed."""
    buf = np.empty(nbytes, np.uint8)
    buf.fill(0)
    return buf


def _check(rc, handle=None):
    if rc != OK:
        msg = lib().coral_last_error(handle)
        raise CoralError(rc, msg.decode() if msg else "")


def default_params() -> Params:
    p = Params()
    _check(lib().coral_params_default(ctypes.byref(p)))
    return p


def params_from_world(world, path=FP32_PERCELL, **overrides) -> Params:
    """Library params for a ``worlds.World`` (its physics constants, hidden size and seed)."""
    p = default_params()
    ph = dict(world.physics)
    p.hidden = world.hidden
    p.path = path
    for k in ("k_inv", "k_liq", "k_exp", "k_flow", "e_day", "e_night", "sigma_mut"):
        setattr(p, k, float(ph[k]))
    p.day_period = int(ph["day_period"])
    p.rotation = int(ph["rotation"])
    p.radiation_every = int(ph.get("radiation_every", 0))
    p.p_mut = float(ph.get("p_mut", 0.0))
    p.p_merge = float(ph.get("p_merge", 0.0))
    p.seed = int(world.seed)
    for k, v in overrides.items():
        setattr(p, k, v)
    return p


def _ptr(a):
    """(pointer, on_device) of a numpy array or a torch tensor; None -> (None, 0)."""
    if a is None:
        return None, 0
    if isinstance(a, np.ndarray):
        if not a.flags["C_CONTIGUOUS"]:
            raise ValueError("arrays must be C-contiguous")
        return a.ctypes.data, 0
    if hasattr(a, "data_ptr"):
        if not a.is_contiguous():
            raise ValueError("tensors must be contiguous")
        return a.data_ptr(), 1 if a.is_cuda else 0
    raise TypeError(f"unsupported array type {type(a)}")


class Substrate:
    """One torus and its genome table on the current CUDA device (library-owned memory)."""

    def __init__(self, params: Params, width: int, height: int, capacity: int, stream=None):
        self.params = params
        self.width, self.height, self.capacity = int(width), int(height), int(capacity)
        self.n = self.width * self.height
        h = ctypes.c_void_p()
        sp = None
        if stream is not None:
            sp = stream.cuda_stream if hasattr(stream, "cuda_stream") else int(stream)
        _check(lib().coral_substrate_create(ctypes.byref(params), self.width, self.height,
                                            self.capacity, sp, ctypes.byref(h)))
        self.h = h
        self._keep = []

    # -- lifetime
    def close(self):
        if getattr(self, "h", None):
            lib().coral_substrate_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    # -- loads
    def load_state(self, E=None, I=None, C=None, G=None, R=None):
        args = [E, I, C, G, R]
        host = [a for a in args if isinstance(a, np.ndarray)]
        conv = []
        for a, dt in zip(args, (np.float32, np.float32, np.float32, np.int32, np.uint8)):
            if isinstance(a, np.ndarray):
                a = np.ascontiguousarray(a, dtype=dt)
            conv.append(a)
        ptrs = [_ptr(a) for a in conv]
        dev = {d for p, d in ptrs if p is not None}
        if len(dev) > 1:
            raise ValueError("mix of host and device arrays in one load")
        _check(lib().coral_state_load(self.h, *[p for p, _ in ptrs], dev.pop() if dev else 0), self.h)
        del host

    def load_world(self, world):
        self.load_state(world.E, world.I, world.C, world.G, world.R)
        self.load_genomes(genes=world.genes, dense=world.dense, n=world.n_genomes)
        if world.genes is not None:
            self.generate_weights()

    def load_genomes(self, genes=None, dense=None, n=None):
        g = None if genes is None else np.ascontiguousarray(genes, np.float32)
        d = None if dense is None else np.ascontiguousarray(dense, np.float32)
        n = int(n if n is not None else (g.shape[0] if g is not None else d.shape[0]))
        _check(lib().coral_genome_table_load(self.h, n, _ptr(g)[0], _ptr(d)[0], 0), self.h)
        self.n_loaded = n

    def generate_weights(self, slots=None):
        if slots is None:
            _check(lib().coral_cppn_generate_weights(self.h, None, self.n_loaded), self.h)
        else:
            s = np.ascontiguousarray(slots, np.int32)
            _check(lib().coral_cppn_generate_weights(self.h, s.ctypes.data, len(s)), self.h)

    # -- stepping
    def step(self, n=1):
        _check(lib().coral_step(self.h, int(n)), self.h)

    def read_perm_only(self):
        """Runs the bucketing sort (coral_read_perm) without copying its results out."""
        _check(lib().coral_read_perm(self.h, None, None), self.h)

    def step_jobs(self, host_in, host_out, n_steps=1, t0=0):
        """Host-to-host stepping of independent states (coral_step_jobs): host_in / host_out
        are equal-length lists of packed-state buffers (29 bytes per cell, CH_ALL order; numpy
        arrays or CPU tensors, ideally pinned). Copies overlap with the steps."""
        if len(host_in) != len(host_out):
            raise ValueError("host_in and host_out must have the same length")
        need = STATE_BYTES * self.n
        ptrs_in, ptrs_out = [], []
        for bufs, ptrs in ((host_in, ptrs_in), (host_out, ptrs_out)):
            for b in bufs:
                p, dev = _ptr(b)
                size = b.nbytes if isinstance(b, np.ndarray) else b.numel() * b.element_size()
                if dev or size < need:
                    raise ValueError(f"job buffers must be host memory of at least {need} bytes")
                ptrs.append(p)
        k = len(ptrs_in)
        arr_in = (_VP * max(k, 1))(*ptrs_in)
        arr_out = (_VP * max(k, 1))(*ptrs_out)
        _check(lib().coral_step_jobs(self.h, k, arr_in, arr_out, int(n_steps), int(t0)), self.h)

    def step_timed(self, n=1):
        """Steps with CUDA-event timing; returns (step_ms [n], stage_ms [n][3])."""
        step_ms = np.empty(int(n), np.float32)
        stage_ms = np.empty((int(n), 3), np.float32)
        _check(lib().coral_step_timed(self.h, int(n), step_ms.ctypes.data, stage_ms.ctypes.data), self.h)
        return step_ms, stage_ms

    def set_step(self, t):
        _check(lib().coral_set_step(self.h, int(t)), self.h)

    def set_fma_cutoff(self, cells):
        """Small-genome path of the BF16 network: later genome rounds of a tile with at most
        ``cells`` cells of their genome run on the CUDA cores (0 = off)."""
        _check(lib().coral_set_fma_cutoff(self.h, int(cells)), self.h)

    def get_step(self):
        t = ctypes.c_int64()
        _check(lib().coral_get_step(self.h, ctypes.byref(t)), self.h)
        return t.value

    def sync(self):
        _check(lib().coral_sync(self.h), self.h)

    def launch_config(self):
        v = (ctypes.c_int32 * 3)()
        _check(lib().coral_launch_config(self.h, ctypes.byref(v, 0), ctypes.byref(v, 4), ctypes.byref(v, 8)), self.h)
        return {"grid_pass1": v[0], "grid_pass2": v[1], "sms": v[2]}

    # -- reads
    def read_channels(self, mask=CH_ALL, out=None):
        """Planes selected by ``mask`` as a dict of host numpy arrays (or into ``out``: a
        device/host buffer of the packed size, returned as is)."""
        n = self.n
        nbytes = sum((n if b == 7 else 4 * n) for b in range(8) if mask & (1 << b))
        if out is not None:
            p, dev = _ptr(out)
            size = out.nbytes if isinstance(out, np.ndarray) else out.numel() * out.element_size()
            _check(lib().coral_read_channels(self.h, mask, p, size, dev), self.h)
            return out
        buf = _touched(nbytes)
        _check(lib().coral_read_channels(self.h, mask, buf.ctypes.data, nbytes, 0), self.h)
        # the planes are views of the one buffer (no further copies); "C" views the four
        # com planes together when all of them were read (they are adjacent in the buffer)
        res, o, off = {}, 0, {}
        names = ["E", "I", "C0", "C1", "C2", "C3", "G", "R"]
        for b in range(8):
            if not mask & (1 << b):
                continue
            off[b] = o
            if b == 7:
                res["R"] = buf[o:o + n].reshape(self.height, self.width)
                o += n
            else:
                dt = np.int32 if b == 6 else np.float32
                res[names[b]] = buf[o:o + 4 * n].view(dt).reshape(self.height, self.width)
                o += 4 * n
        if all(b in off for b in (2, 3, 4, 5)):
            res["C"] = buf[off[2]:off[2] + 16 * n].view(np.float32).reshape(4, self.height, self.width)
        return res

    def read_stats(self, step_from, n=1):
        out = (Stats * n)()
        _check(lib().coral_read_stats(self.h, int(step_from), int(n), out), self.h)
        return [s.as_dict() for s in out]

    def read_perm(self):
        counts = np.empty(self.capacity, np.int32)
        perm = np.empty(self.n, np.int32)
        _check(lib().coral_read_perm(self.h, counts.ctypes.data, perm.ctypes.data), self.h)
        return counts, perm

    def read_genomes(self):
        genes = np.empty((self.capacity, 18), np.float32)
        parent = np.empty(self.capacity, np.int32)
        _check(lib().coral_read_genomes(self.h, genes.ctypes.data, parent.ctypes.data), self.h)
        return genes, parent

    def genome_distances(self, slots):
        """NEAT compatibility distances [n][n] between the listed genome slots."""
        sl = np.ascontiguousarray(slots, np.int32)
        out = np.empty((len(sl), len(sl)), np.float32)
        _check(lib().coral_genome_distances(self.h, sl.ctypes.data, len(sl), out.ctypes.data), self.h)
        return out

    # -- row slabs (see coral_slab_set in include/coral.h)
    def slab_set(self, row_lo, row_hi, global_cell0):
        _check(lib().coral_slab_set(self.h, int(row_lo), int(row_hi), int(global_cell0)), self.h)

    def copy_rows_from(self, dst_row, src, src_row, n_rows):
        _check(lib().coral_copy_rows(self.h, int(dst_row), src.h, int(src_row), int(n_rows)), self.h)

    def slab_totals(self):
        out = np.empty(6, np.float64)
        _check(lib().coral_slab_totals(self.h, out.ctypes.data), self.h)
        return out

    def slab_radiation_scan(self):
        """(live uint8 [capacity], hits int32 [listed][5], counts int32 [4])."""
        live = np.empty(self.capacity, np.uint8)
        hits = np.empty((self.capacity, 5), np.int32)
        counts = np.empty(4, np.int32)
        _check(lib().coral_slab_radiation_scan(self.h, live.ctypes.data, hits.ctypes.data, self.capacity,
                                               counts.ctypes.data), self.h)
        return live, hits[:counts[3]].copy(), counts

    def slab_radiation_apply(self, live_all, hits_all, counts_all):
        live = np.ascontiguousarray(live_all, np.uint8)
        hits = np.ascontiguousarray(hits_all, np.int32).reshape(-1, 5)
        counts = np.ascontiguousarray(counts_all, np.int32)
        _check(lib().coral_slab_radiation_apply(self.h, live.ctypes.data, hits.ctypes.data if len(hits) else None,
                                                len(hits), counts.ctypes.data), self.h)

    def read_weights(self, slot):
        nf = lib().coral_net_floats(self.params.hidden)
        dst = np.empty(nf, np.float32)
        _check(lib().coral_read_weights(self.h, int(slot), dst.ctypes.data, nf), self.h)
        return dst


def net_floats(hidden):
    return lib().coral_net_floats(int(hidden))


def substrate_for_world(world, path=FP32_PERCELL, stream=None, **overrides) -> Substrate:
    """Create a substrate sized for ``world`` and load its state and genome table."""
    s = Substrate(params_from_world(world, path, **overrides), world.width, world.height,
                  world.capacity, stream)
    s.load_world(world)
    return s


def bf16_available() -> bool:
    """True when the library was built with the tcgen05 tensor-core network and the current
    device can run it (probed by creating a minimal BF16-path substrate)."""
    try:
        p = default_params()
        p.path = BF16_GROUPED
        s = Substrate(p, 3, 3, 1)
        s.close()
        return True
    except CoralError:
        return False


NOALLOC_MAX_CELLS = 1 << 20
NOALLOC_MAX_CAPACITY = 1 << 16


def bucket_noalloc(G, capacity, counts, perm, stream=None):
    """Stable counting sort of cell ids by genome slot on caller-owned CUDA tensors, with no
    device allocation (fixed library scratch; see coral_bucket_noalloc in include/coral.h).
    G: int32 [n] (n <= 1,048,576), counts: int32 [capacity] (<= 65,536), perm: int32 [n]."""
    sp = None
    if stream is not None:
        sp = stream.cuda_stream if hasattr(stream, "cuda_stream") else int(stream)
    rc = lib().coral_bucket_noalloc(_ptr(G)[0], int(G.numel()), int(capacity), _ptr(counts)[0],
                                    _ptr(perm)[0], sp)
    if rc != OK:
        raise CoralError(rc, lib().coral_bucket_noalloc_last_error().decode())


class Batch:
    """Many substrates stepped together: one launch per pass over all worlds, each step a CUDA
    graph replay (see coral_batch_create in include/coral.h). The substrates stay owned by
    the caller and must outlive the batch."""

    def __init__(self, substrates):
        self.worlds = list(substrates)
        arr = (ctypes.c_void_p * len(self.worlds))(*[s.h for s in self.worlds])
        h = ctypes.c_void_p()
        rc = lib().coral_batch_create(arr, len(self.worlds), ctypes.byref(h))
        if rc != OK:
            raise CoralError(rc, lib().coral_last_error(None).decode())
        self.h = h

    def _check(self, rc):
        if rc != OK:
            raise CoralError(rc, lib().coral_last_error(None).decode())

    def step(self, n=1):
        self._check(lib().coral_batch_step(self.h, int(n)))

    def step_timed(self, n=1):
        ms = np.empty(int(n), np.float32)
        self._check(lib().coral_batch_step_timed(self.h, int(n), ms.ctypes.data))
        return ms

    def set_fma_cutoff(self, cells):
        self._check(lib().coral_batch_set_fma_cutoff(self.h, int(cells)))

    def tune(self, trial_steps=3):
        c = np.zeros(4, np.int32)
        self._check(lib().coral_batch_tune(self.h, int(trial_steps), c.ctypes.data))
        return {"pass1_ctas_per_sm": int(c[0]), "pass2_ctas_per_sm": int(c[1]), "step_us": int(c[2]),
                "fma_cutoff": int(c[3])}

    def close(self):
        if getattr(self, "h", None):
            lib().coral_batch_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()


def philox4x32_10(ctr, key):
    """Philox4x32-10 evaluated on the device by the radiation kernels' function (test hook):
    ctr uint32 [n][4], key uint32 [n][2] -> uint32 [n][4]."""
    c = np.ascontiguousarray(ctr, np.uint32).reshape(-1, 4)
    k = np.ascontiguousarray(key, np.uint32).reshape(-1, 2)
    if len(c) != len(k):
        raise ValueError("ctr and key must have the same number of rows")
    out = np.empty_like(c)
    _check(lib().coral_philox4x32_10(c.ctypes.data, k.ctypes.data, out.ctypes.data, len(c)))
    return out


def measure_sfu_rate(stream=None) -> float:
    """tanh.approx.f32 evaluations per second of the current device (measurement hook)."""
    v = ctypes.c_double(0.0)
    sp = None if stream is None else (stream.cuda_stream if hasattr(stream, "cuda_stream") else int(stream))
    _check(lib().coral_measure_sfu_rate(sp, ctypes.byref(v)))
    return v.value


def selftest_wait_timeout(wait_us=1000, stream=None):
    """Runs the failure-detection self-test; returns the status the kernel recorded
    (E_TIMEOUT when the bounded wait ran out as designed)."""
    st = ctypes.c_int32(0)
    sp = None if stream is None else (stream.cuda_stream if hasattr(stream, "cuda_stream") else int(stream))
    _check(lib().coral_selftest_wait_timeout(sp, int(wait_us), ctypes.byref(st)))
    return st.value
