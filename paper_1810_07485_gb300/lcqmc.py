"""Thin ctypes binding of liblcqmc.so (include/lcqmc.h).

Argument marshalling only: every step of an update runs in the library's CUDA
kernels.  There is no CPU fallback; loading fails loudly when the library has
not been built.  Streams may come from PyTorch (torch.cuda.Stream.cuda_stream).
"""
import ctypes
import os

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "liblcqmc.so")

OK = 0
PENDING = 1
ERRORS = {-1: "E_INVAL", -2: "E_NOMEM", -3: "E_TOO_LARGE", -4: "E_ID_OVERFLOW",
          -5: "E_DEVICE_TIMEOUT", -6: "E_CUDA", -7: "E_STATE", -8: "E_NOT_FOUND",
          -9: "E_CANCELLED", -10: "E_CAPACITY"}
NPHASE = 8
PHASES = ["insert", "cut", "link_union", "loop_ids", "loop_props", "op_offsets", "op_rewrite", "spin_rewrite"]


class LcqmcError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__(f"{ERRORS.get(code, code)}: {msg}")
        self.code = code


NOBS = 9  # E/L, chi_s, chi(pi+2pi/L), n, n_off, fragments, loops, V+E, chi(pi, 2pi/beta)


class Obs(ctypes.Structure):
    _fields_ = [("n_updates", ctypes.c_int64), ("sum", ctypes.c_double * NOBS),
                ("sumsq", ctypes.c_double * NOBS), ("xi", ctypes.c_double),
                ("xi_tau", ctypes.c_double), ("gap", ctypes.c_double)]


class Tuning(ctypes.Structure):
    _fields_ = [("link_threads", ctypes.c_int32), ("link_x_warps", ctypes.c_int32),
                ("compress_threads", ctypes.c_int32), ("pad", ctypes.c_int32)]

    def as_dict(self):
        return {"link_threads": self.link_threads, "link_x_warps": self.link_x_warps,
                "compress_threads": self.compress_threads}


SW_NOBS = 4  # energy per site, sum_c |c|^2 / N, M^2 / N, |M| / N
SW_NPHASE = 4
SW_PHASES = ("tile_bonds_uf", "boundary_merge", "roots_flip", "open_sizes_record")


class SwObs(ctypes.Structure):
    _fields_ = [("n_updates", ctypes.c_int64), ("sum", ctypes.c_double * SW_NOBS),
                ("sumsq", ctypes.c_double * SW_NOBS)]


SW_RECORD_DTYPE = np.dtype([("sweep", np.int64), ("n_eq", np.int64), ("n_act", np.int64),
                            ("n_clusters", np.int64), ("max_cluster", np.int64), ("sum_c2", np.uint64),
                            ("mag", np.int64), ("energy", np.float64), ("chi", np.float64)])


class Record(ctypes.Structure):
    _fields_ = [("n", ctypes.c_int64), ("n_off_old", ctypes.c_int64), ("n_off_new", ctypes.c_int64),
                ("n_free", ctypes.c_int64), ("n_clusters", ctypes.c_int64), ("n_seg", ctypes.c_int64),
                ("F", ctypes.c_int32), ("pad", ctypes.c_int32),
                ("sw2_lo", ctypes.c_uint64), ("sw2_hi", ctypes.c_uint64),
                ("sf2_lo", ctypes.c_uint64), ("sf2_hi", ctypes.c_uint64),
                ("sz2_lo", ctypes.c_uint64), ("sz2_hi", ctypes.c_uint64),
                ("energy", ctypes.c_double), ("chi_s", ctypes.c_double), ("chi_q", ctypes.c_double),
                ("chi_w", ctypes.c_double)]


RECORD_DTYPE = np.dtype([("n", np.int64), ("n_off_old", np.int64), ("n_off_new", np.int64),
                         ("n_free", np.int64), ("n_clusters", np.int64), ("n_seg", np.int64),
                         ("F", np.int32), ("pad", np.int32), ("sw2_lo", np.uint64),
                         ("sw2_hi", np.uint64), ("sf2_lo", np.uint64), ("sf2_hi", np.uint64),
                         ("sz2_lo", np.uint64), ("sz2_hi", np.uint64),
                         ("energy", np.float64), ("chi_s", np.float64), ("chi_q", np.float64),
                         ("chi_w", np.float64)])
assert RECORD_DTYPE.itemsize == ctypes.sizeof(Record)


class Geometry(ctypes.Structure):
    _fields_ = [("L", ctypes.c_int64), ("nsub", ctypes.c_int64), ("nbond", ctypes.c_int64),
                ("nwin", ctypes.c_int64), ("ncell", ctypes.c_int64), ("Q", ctypes.c_int32),
                ("F", ctypes.c_int32), ("J", ctypes.c_double), ("beta", ctypes.c_double),
                ("w", ctypes.c_double), ("seed", ctypes.c_uint64), ("sweep", ctypes.c_uint32),
                ("replays", ctypes.c_uint32)]


class ChainSpec(ctypes.Structure):
    _fields_ = [("L", ctypes.c_int64), ("S", ctypes.c_double), ("J", ctypes.c_double),
                ("beta", ctypes.c_double), ("seed", ctypes.c_uint64)]


class Request(ctypes.Structure):
    _fields_ = [("L", ctypes.c_int64), ("S", ctypes.c_double), ("J", ctypes.c_double),
                ("beta", ctypes.c_double), ("seed", ctypes.c_uint64), ("n_updates", ctypes.c_int64)]


class Result(ctypes.Structure):
    _fields_ = [("status", ctypes.c_int32), ("pad", ctypes.c_int32), ("obs", Obs),
                ("t_submit", ctypes.c_double), ("t_admit", ctypes.c_double),
                ("t_done", ctypes.c_double), ("vertices_edges", ctypes.c_int64)]


_lib = None


def lib():
    """Loads liblcqmc.so; raises if it was not built (no CPU fallback)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(LIB_PATH):
        raise ImportError(f"{LIB_PATH} not found: build it with paper_1810_07485_gb300.build.build()")
    L = ctypes.CDLL(LIB_PATH)
    vp, i64, u64, i32, u32, dbl = (ctypes.c_void_p, ctypes.c_int64, ctypes.c_uint64, ctypes.c_int,
                                   ctypes.c_uint32, ctypes.c_double)
    P = ctypes.POINTER
    sig = {
        "lcqmc_create": [i64, dbl, dbl, dbl, u64, P(vp)],
        "lcqmc_create_ex": [i64, dbl, dbl, dbl, u64, vp, vp, P(vp)],
        "lcqmc_update": [vp, i64],
        "lcqmc_sync": [vp],
        "lcqmc_measure": [vp, P(Obs)],
        "lcqmc_reset_obs": [vp],
        "lcqmc_get_records": [vp, vp, i64, P(i64)],
        "lcqmc_get_geometry": [vp, P(Geometry)],
        "lcqmc_export_config": [vp, vp, vp, vp, i64, P(i64)],
        "lcqmc_import_config": [vp, vp, vp, vp, i64, u32],
        "lcqmc_set_keep_graph": [vp, i32],
        "lcqmc_export_graph": [vp, vp, vp, vp, vp, vp, i64, P(i64)],
        "lcqmc_export_cells": [vp, vp, i64],
        "lcqmc_checkpoint": [vp, vp, P(ctypes.c_size_t)],
        "lcqmc_restore": [vp, vp, ctypes.c_size_t],
        "lcqmc_set_phase_timing": [vp, i32],
        "lcqmc_set_temporal": [vp, i32],
        "lcqmc_set_wait_limit": [vp, i64],
        "lcqmc_get_tuning": [vp, P(Tuning)],
        "lcqmc_set_tuning": [vp, P(Tuning)],
        "lcqmc_autotune": [vp, i64, P(Tuning)],
        "lcqmc_batch_get_tuning": [vp, P(Tuning)],
        "lcqmc_batch_set_tuning": [vp, P(Tuning)],
        "lcqmc_batch_autotune": [vp, i64, P(Tuning)],
        "lcqmc_get_phase_times": [vp, vp, i32],
        "lcqmc_destroy": [vp],
        "lcqmc_batch_create": [i64, vp, vp, P(vp)],
        "lcqmc_batch_update": [vp, i64],
        "lcqmc_batch_sync": [vp],
        "lcqmc_batch_set_temporal": [vp, i32],
        "lcqmc_batch_measure": [vp, i64, P(Obs)],
        "lcqmc_batch_get_records": [vp, i64, vp, i64, P(i64)],
        "lcqmc_batch_destroy": [vp],
        "lcqmc_server_create": [ctypes.c_size_t, i32, P(vp)],
        "lcqmc_submit": [vp, P(Request), P(u64)],
        "lcqmc_poll": [vp, u64, P(Result)],
        "lcqmc_cancel": [vp, u64],
        "lcqmc_server_destroy": [vp],
        "lcqmc_footprint": [i64, dbl, dbl, dbl, P(ctypes.c_size_t)],
        "lcqmc_selftest": [i32, i64, u64, P(i64)],
        "lcqmc_loops_noalloc": [vp, vp, i64, vp, vp],
        "lcqmc_sw_create": [i64, dbl, u64, vp, P(vp)],
        "lcqmc_sw_update": [vp, i64],
        "lcqmc_sw_sync": [vp],
        "lcqmc_sw_get_records": [vp, vp, i64, P(i64)],
        "lcqmc_sw_measure": [vp, P(SwObs)],
        "lcqmc_sw_set_spins": [vp, vp, u32],
        "lcqmc_sw_get_spins": [vp, vp],
        "lcqmc_sw_get_roots": [vp, vp],
        "lcqmc_sw_set_phase_timing": [vp, i32],
        "lcqmc_sw_get_phase_times": [vp, vp, i32],
        "lcqmc_sw_destroy": [vp],
    }
    for name, args in sig.items():
        f = getattr(L, name)
        f.argtypes = args
        f.restype = ctypes.c_int
    L.lcqmc_last_error.restype = ctypes.c_char_p
    L.lcqmc_last_error.argtypes = []
    L.lcqmc_stream.restype = vp
    L.lcqmc_stream.argtypes = [vp]
    L.lcqmc_sw_stream.restype = vp
    L.lcqmc_sw_stream.argtypes = [vp]
    _lib = L
    return L


def _check(rc):
    if rc < 0:
        raise LcqmcError(rc, lib().lcqmc_last_error().decode())
    return rc


def _p(a):
    return None if a is None else a.ctypes.data_as(ctypes.c_void_p)


def u128(lo, hi):
    return (int(hi) << 64) | int(lo)


def records_to_numpy(buf, n):
    return np.frombuffer(bytes(buf), dtype=RECORD_DTYPE, count=n).copy()


class Chain:
    """One Markov chain on the GPU: lcqmc_create ... lcqmc_destroy."""

    def __init__(self, L, beta, S=0.5, J=1.0, seed=1, stream=None):
        h = ctypes.c_void_p()
        if stream is None:
            _check(lib().lcqmc_create(int(L), float(S), float(J), float(beta), int(seed) & (2**64 - 1),
                                      ctypes.byref(h)))
        else:
            _check(lib().lcqmc_create_ex(int(L), float(S), float(J), float(beta),
                                         int(seed) & (2**64 - 1), ctypes.c_void_p(int(stream)), None,
                                         ctypes.byref(h)))
        self.h = h
        self.L, self.beta, self.S, self.J, self.seed = int(L), float(beta), float(S), float(J), int(seed)

    def close(self):
        if self.h:
            lib().lcqmc_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()

    @property
    def stream(self):
        return lib().lcqmc_stream(self.h)

    def update(self, n=1):
        _check(lib().lcqmc_update(self.h, int(n)))

    def sync(self):
        _check(lib().lcqmc_sync(self.h))

    def measure(self):
        o = Obs()
        _check(lib().lcqmc_measure(self.h, ctypes.byref(o)))
        return o

    def reset_obs(self):
        _check(lib().lcqmc_reset_obs(self.h))

    def records(self, max_n=1 << 16):
        buf = (Record * max(1, max_n))()
        cnt = ctypes.c_int64()
        _check(lib().lcqmc_get_records(self.h, buf, int(max_n), ctypes.byref(cnt)))
        return records_to_numpy(buf, cnt.value)

    def geometry(self):
        g = Geometry()
        _check(lib().lcqmc_get_geometry(self.h, ctypes.byref(g)))
        return g

    def export_config(self):
        g = self.geometry()
        n = ctypes.c_int64()
        _check(lib().lcqmc_export_config(self.h, None, None, None, 0, ctypes.byref(n)))
        s0 = np.zeros(g.nsub, np.uint8)
        ptr = np.zeros(g.ncell + 1, np.int32)
        tau = np.zeros(max(1, n.value), np.float64)
        _check(lib().lcqmc_export_config(self.h, _p(s0), _p(ptr), _p(tau), n.value, ctypes.byref(n)))
        return s0, ptr, tau[: n.value].copy()

    def import_config(self, s0, op_ptr, op_tau, sweep):
        s0 = np.ascontiguousarray(s0, np.uint8)
        op_ptr = np.ascontiguousarray(op_ptr, np.int32)
        op_tau = np.ascontiguousarray(op_tau, np.float64)
        _check(lib().lcqmc_import_config(self.h, _p(s0), _p(op_ptr), _p(op_tau) if len(op_tau) else None,
                                         len(op_tau), int(sweep)))

    def export_graph(self, fields=("tau", "flag", "pl", "pr", "root")):
        n = ctypes.c_int64()
        _check(lib().lcqmc_export_graph(self.h, None, None, None, None, None, 0, ctypes.byref(n)))
        m = n.value
        dt = dict(tau=np.float64, flag=np.uint8, pl=np.int32, pr=np.int32, root=np.int32)
        out = {k: np.zeros(m, dt[k]) for k in fields}
        args = [_p(out.get(k)) for k in ("tau", "flag", "pl", "pr", "root")]
        _check(lib().lcqmc_export_graph(self.h, *args, m, ctypes.byref(n)))
        return out

    def export_cells(self):
        g = self.geometry()
        v = np.zeros(g.ncell + 1, np.int32)
        _check(lib().lcqmc_export_cells(self.h, _p(v), g.ncell + 1))
        return v

    def checkpoint(self):
        ln = ctypes.c_size_t()
        _check(lib().lcqmc_checkpoint(self.h, None, ctypes.byref(ln)))
        buf = (ctypes.c_char * ln.value)()
        _check(lib().lcqmc_checkpoint(self.h, buf, ctypes.byref(ln)))
        return bytes(buf[: ln.value])

    def restore(self, blob):
        buf = ctypes.create_string_buffer(blob, len(blob))
        _check(lib().lcqmc_restore(self.h, buf, len(blob)))

    def set_phase_timing(self, on=True):
        _check(lib().lcqmc_set_phase_timing(self.h, 1 if on else 0))

    def set_wait_limit(self, limit=0):
        _check(lib().lcqmc_set_wait_limit(self.h, int(limit)))

    def set_temporal(self, on=True):
        """Temporal moment chi(pi, 2 pi / beta) on or off (off after create)."""
        _check(lib().lcqmc_set_temporal(self.h, 1 if on else 0))

    def tuning(self):
        t = Tuning()
        _check(lib().lcqmc_get_tuning(self.h, ctypes.byref(t)))
        return t.as_dict()

    def set_tuning(self, link_threads=256, link_x_warps=8, compress_threads=128):
        _check(lib().lcqmc_set_tuning(self.h, ctypes.byref(Tuning(link_threads, link_x_warps,
                                                                  compress_threads, 0))))

    def autotune(self, updates_per_trial=2):
        t = Tuning()
        _check(lib().lcqmc_autotune(self.h, int(updates_per_trial), ctypes.byref(t)))
        return t.as_dict()

    def phase_times(self):
        ms = np.zeros(NPHASE)
        _check(lib().lcqmc_get_phase_times(self.h, _p(ms), NPHASE))
        return dict(zip(PHASES, ms))


class Batch:
    """Many independent chains updated together (lcqmc_batch_*)."""

    def __init__(self, specs, stream=None):
        arr = (ChainSpec * len(specs))()
        for i, s in enumerate(specs):
            arr[i] = ChainSpec(int(s["L"]), float(s.get("S", 0.5)), float(s.get("J", 1.0)),
                               float(s["beta"]), int(s.get("seed", i)) & (2**64 - 1))
        h = ctypes.c_void_p()
        _check(lib().lcqmc_batch_create(len(specs), arr, ctypes.c_void_p(int(stream)) if stream else None,
                                        ctypes.byref(h)))
        self.h = h
        self.n = len(specs)

    def close(self):
        if self.h:
            lib().lcqmc_batch_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def update(self, n=1):
        _check(lib().lcqmc_batch_update(self.h, int(n)))

    def sync(self):
        _check(lib().lcqmc_batch_sync(self.h))

    def set_temporal(self, on=True):
        _check(lib().lcqmc_batch_set_temporal(self.h, 1 if on else 0))

    def tuning(self):
        t = Tuning()
        _check(lib().lcqmc_batch_get_tuning(self.h, ctypes.byref(t)))
        return t.as_dict()

    def set_tuning(self, link_threads=256, link_x_warps=8, compress_threads=128):
        _check(lib().lcqmc_batch_set_tuning(self.h, ctypes.byref(Tuning(link_threads, link_x_warps,
                                                                        compress_threads, 0))))

    def autotune(self, updates_per_trial=1):
        t = Tuning()
        _check(lib().lcqmc_batch_autotune(self.h, int(updates_per_trial), ctypes.byref(t)))
        return t.as_dict()

    def measure(self, i):
        o = Obs()
        _check(lib().lcqmc_batch_measure(self.h, int(i), ctypes.byref(o)))
        return o

    def records(self, i, max_n=1 << 12):
        buf = (Record * max(1, max_n))()
        cnt = ctypes.c_int64()
        _check(lib().lcqmc_batch_get_records(self.h, int(i), buf, int(max_n), ctypes.byref(cnt)))
        return records_to_numpy(buf, cnt.value)


def footprint(L, beta, S=0.5, J=1.0):
    """Device bytes one served chain holds (host-only computation)."""
    b = ctypes.c_size_t()
    _check(lib().lcqmc_footprint(int(L), float(S), float(J), float(beta), ctypes.byref(b)))
    return b.value


class Server:
    """Served form: continuous batching of simulation requests (lcqmc_server_*)."""

    def __init__(self, hbm_budget, max_slots):
        h = ctypes.c_void_p()
        _check(lib().lcqmc_server_create(int(hbm_budget), int(max_slots), ctypes.byref(h)))
        self.h = h

    def close(self):
        if self.h:
            lib().lcqmc_server_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def submit(self, L, beta, n_updates, S=0.5, J=1.0, seed=1):
        """Returns a ticket, or raises LcqmcError (E_TOO_LARGE, E_ID_OVERFLOW, ...)."""
        r = Request(int(L), float(S), float(J), float(beta), int(seed) & (2**64 - 1), int(n_updates))
        t = ctypes.c_uint64()
        _check(lib().lcqmc_submit(self.h, ctypes.byref(r), ctypes.byref(t)))
        return t.value

    def poll(self, ticket):
        """None while pending, else the Result (status, obs, timestamps)."""
        res = Result()
        rc = _check(lib().lcqmc_poll(self.h, int(ticket), ctypes.byref(res)))
        return None if rc == PENDING else res

    def cancel(self, ticket):
        _check(lib().lcqmc_cancel(self.h, int(ticket)))


class SWIsing:
    """Swendsen-Wang updates of the L x L periodic Ising model (lcqmc_sw_*)."""

    def __init__(self, L, K, seed=1, stream=None):
        h = ctypes.c_void_p()
        _check(lib().lcqmc_sw_create(int(L), float(K), int(seed) & (2**64 - 1),
                                     ctypes.c_void_p(int(stream)) if stream else None, ctypes.byref(h)))
        self.h = h
        self.L, self.K, self.seed = int(L), float(K), int(seed)

    def close(self):
        if self.h:
            lib().lcqmc_sw_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def update(self, n=1):
        _check(lib().lcqmc_sw_update(self.h, int(n)))

    def sync(self):
        _check(lib().lcqmc_sw_sync(self.h))

    def records(self, max_n=4096):
        buf = np.zeros(max(1, max_n), dtype=SW_RECORD_DTYPE)
        cnt = ctypes.c_int64()
        _check(lib().lcqmc_sw_get_records(self.h, _p(buf), int(max_n), ctypes.byref(cnt)))
        return buf[: cnt.value].copy()

    def measure(self):
        o = SwObs()
        _check(lib().lcqmc_sw_measure(self.h, ctypes.byref(o)))
        return o

    def set_spins(self, spins, sweep=0):
        a = np.ascontiguousarray(spins, dtype=np.uint8).reshape(-1)
        assert a.size == self.L * self.L
        _check(lib().lcqmc_sw_set_spins(self.h, _p(a), ctypes.c_uint32(int(sweep))))

    def spins(self):
        a = np.zeros(self.L * self.L, np.uint8)
        _check(lib().lcqmc_sw_get_spins(self.h, _p(a)))
        return a

    def roots(self):
        a = np.zeros(self.L * self.L, np.int32)
        _check(lib().lcqmc_sw_get_roots(self.h, _p(a)))
        return a

    def set_phase_timing(self, on=True):
        _check(lib().lcqmc_sw_set_phase_timing(self.h, 1 if on else 0))

    def phase_times(self):
        ms = np.zeros(SW_NPHASE)
        _check(lib().lcqmc_sw_get_phase_times(self.h, _p(ms), SW_NPHASE))
        return dict(zip(SW_PHASES, ms.tolist()))

    def stream(self):
        return lib().lcqmc_sw_stream(self.h)
