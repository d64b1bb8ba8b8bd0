"""ctypes binding of the C oracle (test infrastructure).

Only the tests, the smoke entry point and the benchmark's CPU-baseline leg use
this module.  It loads oracle/liboracle.so (built by oracle/build.py) and exposes
the keyed update, the paper-literal serial update, Philox and the Poisson
thresholds on numpy arrays.
"""
import ctypes
import os

import numpy as np

from . import build as _build

KMAX = 48
TW = 4

_lib = None


class Params(ctypes.Structure):
    _fields_ = [("L", ctypes.c_int64), ("Q", ctypes.c_int), ("J", ctypes.c_double),
                ("beta", ctypes.c_double), ("seed", ctypes.c_uint64)]


class Record(ctypes.Structure):
    _fields_ = [("n", ctypes.c_int64), ("n_off_old", ctypes.c_int64),
                ("n_off_new", ctypes.c_int64), ("n_free", ctypes.c_int64),
                ("n_clusters", ctypes.c_int64), ("n_seg", ctypes.c_int64),
                ("F", ctypes.c_int32), ("pad", ctypes.c_int32),
                ("sw2_lo", ctypes.c_uint64), ("sw2_hi", ctypes.c_uint64),
                ("sf2_lo", ctypes.c_uint64), ("sf2_hi", ctypes.c_uint64),
                ("sz2_lo", ctypes.c_uint64), ("sz2_hi", ctypes.c_uint64),
                ("energy", ctypes.c_double), ("chi_s", ctypes.c_double),
                ("chi_q", ctypes.c_double), ("chi_w", ctypes.c_double)]


RECORD_DTYPE = np.dtype([(name, np.int64 if t in (ctypes.c_int64,) else
                          np.uint64 if t is ctypes.c_uint64 else
                          np.int32 if t is ctypes.c_int32 else np.float64)
                         for name, t in Record._fields_])
assert RECORD_DTYPE.itemsize == ctypes.sizeof(Record)


class SwRecord(ctypes.Structure):
    _fields_ = [("n_eq", ctypes.c_int64), ("n_act", ctypes.c_int64),
                ("n_clusters", ctypes.c_int64), ("max_cluster", ctypes.c_int64),
                ("sum_c2", ctypes.c_uint64), ("mag", ctypes.c_int64),
                ("energy", ctypes.c_double), ("chi", ctypes.c_double)]


SW_RECORD_DTYPE = np.dtype([("n_eq", np.int64), ("n_act", np.int64), ("n_clusters", np.int64),
                            ("max_cluster", np.int64), ("sum_c2", np.uint64), ("mag", np.int64),
                            ("energy", np.float64), ("chi", np.float64)])
assert SW_RECORD_DTYPE.itemsize == ctypes.sizeof(SwRecord)


def lib():
    global _lib
    if _lib is None:
        path = _build.build()
        L = ctypes.CDLL(path)
        P = ctypes.POINTER
        vp = ctypes.c_void_p
        L.orc_philox4x32_10.argtypes = [vp, vp, vp]
        L.orc_poisson_thresholds.argtypes = [ctypes.c_double, vp]
        for fn in ("orc_nsub", "orc_nbond", "orc_nwin", "orc_ncell"):
            getattr(L, fn).argtypes = [P(Params)]
            getattr(L, fn).restype = ctypes.c_int64
        L.orc_cell_index.argtypes = [P(Params), ctypes.c_int64, ctypes.c_int64]
        L.orc_cell_index.restype = ctypes.c_int64
        L.orc_fixed_exponent.argtypes = [P(Params)]
        L.orc_fixed_exponent.restype = ctypes.c_int
        L.orc_neel.argtypes = [P(Params), vp, vp]
        L.orc_keyed_update.argtypes = [P(Params), ctypes.c_uint32, vp, vp, vp, vp, vp, vp,
                                       ctypes.c_int64, vp, ctypes.c_int64, vp, vp, vp, vp, vp,
                                       vp]
        L.orc_keyed_update.restype = ctypes.c_int
        L.orc_keyed_run.argtypes = [P(Params), ctypes.c_uint32, ctypes.c_int64, vp, vp, vp,
                                    ctypes.c_int64, vp]
        L.orc_keyed_run.restype = ctypes.c_int
        L.orc_serial_run.argtypes = [P(Params), ctypes.c_uint32, ctypes.c_int64, vp, vp, vp,
                                     vp, ctypes.c_int64, vp]
        L.orc_serial_run.restype = ctypes.c_int
        L.orc_phase.argtypes = [ctypes.c_uint64, ctypes.c_uint64, ctypes.c_int, P(ctypes.c_int64),
                                P(ctypes.c_int64)]
        L.orc_phase_recip.argtypes = [ctypes.c_int64, P(ctypes.c_int)]
        L.orc_phase_recip.restype = ctypes.c_uint64
        L.orc_sw_threshold.argtypes = [ctypes.c_double]
        L.orc_sw_threshold.restype = ctypes.c_uint64
        L.orc_sw_update.argtypes = [ctypes.c_int64, ctypes.c_double, ctypes.c_uint64, ctypes.c_uint32,
                                    vp, vp, vp, P(SwRecord)]
        L.orc_sw_update.restype = ctypes.c_int
        L.orc_sw_run.argtypes = [ctypes.c_int64, ctypes.c_double, ctypes.c_uint64, ctypes.c_uint32,
                                 ctypes.c_int64, vp, vp]
        L.orc_sw_run.restype = ctypes.c_int
        _lib = L
    return _lib


def _ptr(a):
    return a.ctypes.data_as(ctypes.c_void_p)


def params(L, beta, J=1.0, Q=1, seed=1):
    return Params(int(L), int(Q), float(J), float(beta), int(seed) & 0xFFFFFFFFFFFFFFFF)


def philox(ctr, key):
    c = np.ascontiguousarray(ctr, dtype=np.uint32)
    k = np.ascontiguousarray(key, dtype=np.uint32)
    out = np.zeros(4, dtype=np.uint32)
    lib().orc_philox4x32_10(_ptr(c), _ptr(k), _ptr(out))
    return out


def poisson_thresholds(mu):
    T = np.zeros(KMAX, dtype=np.uint64)
    lib().orc_poisson_thresholds(ctypes.c_double(mu), _ptr(T))
    return T


def geometry(p):
    l = lib()
    return dict(nsub=l.orc_nsub(ctypes.byref(p)), nbond=l.orc_nbond(ctypes.byref(p)),
                nwin=l.orc_nwin(ctypes.byref(p)), ncell=l.orc_ncell(ctypes.byref(p)),
                F=l.orc_fixed_exponent(ctypes.byref(p)))


def cell_index(p, b, j):
    return lib().orc_cell_index(ctypes.byref(p), int(b), int(j))


class State:
    """World-line state in the canonical cell layout: s0[nsub] and a CSR of
    off-diagonal operator times per (bond, window) cell."""

    def __init__(self, s0, op_ptr, op_tau):
        self.s0 = np.ascontiguousarray(s0, dtype=np.uint8)
        self.op_ptr = np.ascontiguousarray(op_ptr, dtype=np.int64)
        self.op_tau = np.ascontiguousarray(op_tau, dtype=np.float64)

    def copy(self):
        return State(self.s0.copy(), self.op_ptr.copy(), self.op_tau.copy())


def neel(p):
    g = geometry(p)
    s0 = np.zeros(g["nsub"], dtype=np.uint8)
    ptr = np.zeros(g["ncell"] + 1, dtype=np.int64)
    lib().orc_neel(ctypes.byref(p), _ptr(s0), _ptr(ptr))
    return State(s0, ptr, np.zeros(0, dtype=np.float64))


def keyed_update(p, sweep, st, graph=False, op_cap=None):
    """One keyed update.  Returns (new_state, record, graph_dict_or_None)."""
    g = geometry(p)
    n_old = int(st.op_ptr[-1])
    cap = op_cap if op_cap is not None else max(1024, 4 * n_old + int(2 * p.L * p.Q * p.Q * p.beta) + 64)
    s1 = np.zeros(g["nsub"], dtype=np.uint8)
    p1 = np.zeros(g["ncell"] + 1, dtype=np.int64)
    t1 = np.zeros(cap, dtype=np.float64)
    rec = Record()
    gr = None
    args_g = [ctypes.c_int64(0)] + [None] * 6
    if graph:
        vcap = cap
        gr = dict(tau=np.zeros(vcap), flag=np.zeros(vcap, np.uint8), bond=np.zeros(vcap, np.int64),
                  pl=np.zeros(vcap, np.int64), pr=np.zeros(vcap, np.int64),
                  root=np.zeros(vcap, np.int64))
        args_g = [ctypes.c_int64(vcap)] + [_ptr(gr[k]) for k in ("tau", "flag", "bond", "pl", "pr", "root")]
    rc = lib().orc_keyed_update(ctypes.byref(p), ctypes.c_uint32(sweep), _ptr(st.s0),
                                _ptr(st.op_ptr), _ptr(st.op_tau), _ptr(s1), _ptr(p1), _ptr(t1),
                                ctypes.c_int64(cap), ctypes.byref(rec), *args_g)
    if rc != 0:
        raise RuntimeError(f"orc_keyed_update failed: {rc}")
    new = State(s1, p1, t1[: int(p1[-1])].copy())
    r = record_to_numpy([rec])[0]
    if graph:
        n = int(r["n"])
        gr = {k: v[:n].copy() for k, v in gr.items()}
    return new, r, gr


def record_to_numpy(recs):
    arr = np.zeros(len(recs), dtype=RECORD_DTYPE)
    for i, r in enumerate(recs):
        arr[i] = tuple(getattr(r, f) for f, _ in Record._fields_)
    return arr


def keyed_run(p, sweep0, n_updates, st, op_cap=None):
    """n keyed updates in place on st; returns the records (numpy structured)."""
    n_old = int(st.op_ptr[-1])
    cap = op_cap if op_cap is not None else max(4096, 4 * n_old + int(2 * p.L * p.Q * p.Q * p.beta) + 64)
    tau = np.zeros(cap, dtype=np.float64)
    tau[:n_old] = st.op_tau
    recs = (Record * max(1, n_updates))()
    rc = lib().orc_keyed_run(ctypes.byref(p), ctypes.c_uint32(sweep0), ctypes.c_int64(n_updates),
                             _ptr(st.s0), _ptr(st.op_ptr), _ptr(tau), ctypes.c_int64(cap), recs)
    if rc != 0:
        raise RuntimeError(f"orc_keyed_run failed: {rc}")
    st.op_tau = tau[: int(st.op_ptr[-1])].copy()
    return np.frombuffer(bytes(recs), dtype=RECORD_DTYPE, count=n_updates).copy()


def serial_run(p, sweep0, n_updates, s0=None, ops=None):
    """n paper-literal serial updates starting from (s0, ops) (default Neel, no
    operators).  Returns (records, s0, (tau, bond))."""
    g = geometry(p)
    if s0 is None:
        s0 = (np.arange(g["nsub"]) // p.Q & 1).astype(np.uint8)
    s0 = np.ascontiguousarray(s0, dtype=np.uint8).copy()
    cap = max(4096, int(3 * p.L * p.Q * p.Q * p.beta) + 1024)
    tau = np.zeros(cap)
    bond = np.zeros(cap, dtype=np.int64)
    n_ops = ctypes.c_int64(0)
    if ops is not None:
        n_ops.value = len(ops[0])
        tau[: n_ops.value] = ops[0]
        bond[: n_ops.value] = ops[1]
    recs = (Record * max(1, n_updates))()
    rc = lib().orc_serial_run(ctypes.byref(p), ctypes.c_uint32(sweep0), ctypes.c_int64(n_updates),
                              _ptr(s0), ctypes.byref(n_ops), _ptr(tau), _ptr(bond),
                              ctypes.c_int64(cap), recs)
    if rc != 0:
        raise RuntimeError(f"orc_serial_run failed: {rc}")
    r = np.frombuffer(bytes(recs), dtype=RECORD_DTYPE, count=n_updates).copy()
    return r, s0, (tau[: n_ops.value].copy(), bond[: n_ops.value].copy())


def u128(lo, hi):
    return (int(hi) << 64) | int(lo)


def keyed_cell(p, sweep, st, b, j):
    """Labeling of one cell of the keyed update from state st: (tau, flag)."""
    L = lib()
    if not hasattr(L, "_cell_sig"):
        L.orc_keyed_cell.argtypes = [ctypes.POINTER(Params), ctypes.c_uint32, ctypes.c_void_p,
                                     ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int64, ctypes.c_int64,
                                     ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int64,
                                     ctypes.POINTER(ctypes.c_int64)]
        L.orc_keyed_cell.restype = ctypes.c_int
        L._cell_sig = True
    cap = 4096
    tau = np.zeros(cap)
    flag = np.zeros(cap, np.uint8)
    n = ctypes.c_int64()
    rc = L.orc_keyed_cell(ctypes.byref(p), ctypes.c_uint32(sweep), _ptr(st.s0), _ptr(st.op_ptr),
                          _ptr(st.op_tau), int(b), int(j), _ptr(tau), _ptr(flag), cap, ctypes.byref(n))
    if rc != 0:
        raise RuntimeError("orc_keyed_cell failed")
    return tau[: n.value].copy(), flag[: n.value].copy()


def phase(q, qbeta):
    """exp(i 2 pi q / qbeta) in units of 2^-30 as the oracle evaluates it."""
    c, sn, sh = ctypes.c_int64(), ctypes.c_int64(), ctypes.c_int()
    rb = lib().orc_phase_recip(int(qbeta), ctypes.byref(sh))
    lib().orc_phase(int(q) & (2**64 - 1), rb, sh.value, ctypes.byref(c), ctypes.byref(sn))
    return c.value, sn.value


# ---- Swendsen-Wang 2D Ising (Sec. 4.1 benchmark) ---------------------------------
def sw_threshold(K):
    return int(lib().orc_sw_threshold(float(K)))


def sw_update(L, K, seed, sweep, s, roots=False, bonds=False):
    """One Swendsen-Wang update in place on s (uint8, L*L, row-major).
    Returns (record, roots or None, bonds or None)."""
    assert s.dtype == np.uint8 and s.flags.c_contiguous and s.size == L * L
    rt = np.zeros(L * L, np.int64) if roots else None
    bd = np.zeros(2 * L * L, np.uint8) if bonds else None
    rec = SwRecord()
    rc = lib().orc_sw_update(int(L), float(K), int(seed) & 0xFFFFFFFFFFFFFFFF, ctypes.c_uint32(sweep),
                             _ptr(s), None if rt is None else _ptr(rt), None if bd is None else _ptr(bd),
                             ctypes.byref(rec))
    if rc != 0:
        raise RuntimeError(f"orc_sw_update failed: {rc}")
    r = np.frombuffer(bytes(rec), dtype=SW_RECORD_DTYPE, count=1)[0]
    return r, rt, bd


def sw_run(L, K, seed, sweep0, n, s):
    """n updates in place on s; returns the records."""
    assert s.dtype == np.uint8 and s.flags.c_contiguous and s.size == L * L
    recs = (SwRecord * max(1, n))()
    rc = lib().orc_sw_run(int(L), float(K), int(seed) & 0xFFFFFFFFFFFFFFFF, ctypes.c_uint32(sweep0),
                          int(n), _ptr(s), recs)
    if rc != 0:
        raise RuntimeError(f"orc_sw_run failed: {rc}")
    return np.frombuffer(bytes(recs), dtype=SW_RECORD_DTYPE, count=n).copy()
