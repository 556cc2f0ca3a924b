"""Python binding of the plain CPU oracle (test infrastructure only).

Only the tests, ``__graft_entry__.smoke()`` and the CPU-baseline leg of
``bench.py`` import this module. The product library never calls it.

The oracle computes the truncated local trace of Sec. III (steps 3-8) with
exact dense block exponentials in (n_up, n_dn) sectors, in FP64
(``precision="f64"``) or in the long-double twin of the same C source
(``precision="ext"``). The move editing of a local update (insertion or
removal of a c^+/c pair of one flavor, Sec. II after Eq. (weight_strong))
is written out here with plain Python lists.
"""
from __future__ import annotations

import ctypes
import math
import os
import subprocess
from dataclasses import dataclass

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "kt_oracle.c")
_LIB = os.path.join(_HERE, "libkt_oracle.so")


def build(force: bool = False) -> str:
    """Compile the C oracle (FP64 and long-double twins) into one shared library."""
    if not force and os.path.exists(_LIB) and os.path.getmtime(_LIB) >= os.path.getmtime(_SRC):
        return _LIB
    objs = []
    for real, prefix in (("double", "or64_"), ("long double", "orx_")):
        obj = os.path.join(_HERE, f"_{prefix}o.o")
        subprocess.check_call([
            "gcc", "-O2", "-fPIC", "-fopenmp", "-std=c11", "-c", _SRC, "-o", obj,
            f"-DOR_REAL={real}", f"-DOR_PREFIX={prefix}",
        ])
        objs.append(obj)
    tmp = _LIB + f".tmp{os.getpid()}"
    subprocess.check_call(["gcc", "-shared", "-fopenmp", *objs, "-o", tmp, "-lm"])
    os.replace(tmp, _LIB)
    for o in objs:
        os.remove(o)
    return _LIB


_lib = None


def _load():
    global _lib
    if _lib is None:
        _lib = ctypes.CDLL(build())
        for p in ("or64_", "orx_"):
            getattr(_lib, p + "model_create").argtypes = [
                ctypes.c_int, ctypes.c_double, ctypes.c_double, ctypes.c_double, ctypes.c_double,
                ctypes.c_void_p, ctypes.c_double, ctypes.c_double, ctypes.c_double, ctypes.c_int,
                ctypes.POINTER(ctypes.c_void_p)]
            getattr(_lib, p + "model_free").argtypes = [ctypes.c_void_p]
            getattr(_lib, p + "model_free").restype = None
            getattr(_lib, p + "model_dims").argtypes = [ctypes.c_void_p] + [ctypes.c_void_p] * 4
            getattr(_lib, p + "model_sectors").argtypes = [ctypes.c_void_p] * 3
            getattr(_lib, p + "model_block").argtypes = [ctypes.c_void_p, ctypes.c_int] + [ctypes.c_void_p] * 3
            getattr(_lib, p + "model_kept").argtypes = [ctypes.c_void_p] * 4
            getattr(_lib, p + "trace_batch").argtypes = [ctypes.c_void_p, ctypes.c_int] + [ctypes.c_void_p] * 8 + [ctypes.c_int]
            getattr(_lib, p + "trace_op_batch").argtypes = (
                [ctypes.c_void_p, ctypes.c_int] + [ctypes.c_void_p] * 4 + [ctypes.c_double]
                + [ctypes.c_void_p] * 4 + [ctypes.c_int])
            getattr(_lib, p + "trace_obs_batch").argtypes = (
                [ctypes.c_void_p, ctypes.c_int] + [ctypes.c_void_p] * 4 + [ctypes.c_double, ctypes.c_int]
                + [ctypes.c_void_p] * 4 + [ctypes.c_int])
    return _lib


def _ptr(a: np.ndarray):
    return a.ctypes.data_as(ctypes.c_void_p)


@dataclass
class Params:
    """Model parameters of Eq. (H_loc) plus the truncation of Sec. III."""
    n_orb: int
    U: float
    J: float
    Up: float | None = None  # None -> U - 2J (rotational invariance, Sec. IV.A)
    mu: float = 0.0
    delta: tuple = ()
    beta: float = 10.0
    trunc_eps: float = 1e-10
    deg_tol: float = 1e-9
    density_only: bool = False

    def up(self) -> float:
        return self.U - 2.0 * self.J if self.Up is None else self.Up

    def delta_array(self) -> np.ndarray:
        d = np.zeros(self.n_orb, dtype=np.float64)
        if len(self.delta):
            d[:] = np.asarray(self.delta, dtype=np.float64)
        return d


class Model:
    """Oracle model: dense (n_up, n_dn) blocks, spectrum, kept multiplets."""

    def __init__(self, p: Params, precision: str = "f64"):
        lib = _load()
        self.p = p
        self.prefix = {"f64": "or64_", "ext": "orx_"}[precision]
        self._delta = p.delta_array()
        h = ctypes.c_void_p()
        rc = getattr(lib, self.prefix + "model_create")(
            p.n_orb, p.U, p.J, p.up(), p.mu, _ptr(self._delta), p.beta, p.trunc_eps, p.deg_tol,
            1 if p.density_only else 0, ctypes.byref(h))
        if rc != 0:
            raise RuntimeError(f"oracle model_create failed ({rc})")
        self._h = h
        ns, nsec, nk = ctypes.c_int(), ctypes.c_int(), ctypes.c_int()
        e0 = ctypes.c_double()
        getattr(lib, self.prefix + "model_dims")(h, ctypes.byref(ns), ctypes.byref(nsec), ctypes.byref(nk), ctypes.byref(e0))
        self.nstates, self.nsec, self.nkept, self.E0 = ns.value, nsec.value, nk.value, e0.value
        self.sec_dim = np.zeros(self.nsec, dtype=np.int32)
        self.states = np.zeros(self.nstates, dtype=np.int32)
        getattr(lib, self.prefix + "model_sectors")(h, _ptr(self.sec_dim), _ptr(self.states))
        self.kept_sec = np.zeros(self.nkept, dtype=np.int32)
        self.kept_col = np.zeros(self.nkept, dtype=np.int32)
        self.kept_E = np.zeros(self.nkept, dtype=np.float64)
        getattr(lib, self.prefix + "model_kept")(h, _ptr(self.kept_sec), _ptr(self.kept_col), _ptr(self.kept_E))

    def __del__(self):
        h = getattr(self, "_h", None)
        if h is not None and _lib is not None:
            getattr(_lib, self.prefix + "model_free")(h)
            self._h = None

    def sector_index(self, n_up: int, n_dn: int) -> int:
        return n_up * (self.p.n_orb + 1) + n_dn

    def block(self, s: int):
        """(H, eigenvalues, eigenvectors) of sector s as float64 arrays."""
        d = int(self.sec_dim[s])
        H = np.zeros((d, d)); w = np.zeros(d); V = np.zeros((d, d))
        getattr(_lib, self.prefix + "model_block")(self._h, s, _ptr(H), _ptr(w), _ptr(V))
        return H, w, V

    def sector_states(self, s: int) -> np.ndarray:
        off = int(self.sec_dim[:s].sum())
        return self.states[off: off + int(self.sec_dim[s])]

    def spectrum(self) -> np.ndarray:
        """All eigenvalues, sorted ascending."""
        return np.sort(np.concatenate([self.block(s)[1] for s in range(self.nsec)]))

    def trace(self, seqs: "SeqBatch", nthreads: int = 0):
        """(sign int8, log|T| float64, log|T~| float64) per sequence; raises on invalid input."""
        n = seqs.n
        sign = np.zeros(n, dtype=np.int32)
        la = np.zeros(n, dtype=np.float64)
        lt = np.zeros(n, dtype=np.float64)
        st = np.zeros(n, dtype=np.int32)
        used = getattr(_lib, self.prefix + "trace_batch")(
            self._h, n, _ptr(seqs.offsets), _ptr(seqs.tau), _ptr(seqs.flavor), _ptr(seqs.dagger),
            _ptr(sign), _ptr(la), _ptr(lt), _ptr(st), int(nthreads))
        self.threads_used = used
        if st.any():
            raise ValueError(f"oracle rejected {int((st != 0).sum())} sequences (first at {int(np.argmax(st != 0))})")
        return sign.astype(np.int8), la, lt


    def trace_op(self, seqs: "SeqBatch", t_obs: float, op: np.ndarray, nthreads: int = 0):
        """Traces with a general operator (dense [4^n, 4^n], <y|O|x> at [y, x], conserving
        (n_up, n_dn)) inserted at t_obs. Returns (sign int8 [n], log|T_O| [n])."""
        op = np.ascontiguousarray(op, dtype=np.float64)
        assert op.shape == (self.nstates, self.nstates)
        n = seqs.n
        sign = np.zeros(n, dtype=np.int32)
        la = np.zeros(n, dtype=np.float64)
        st = np.zeros(n, dtype=np.int32)
        getattr(_lib, self.prefix + "trace_op_batch")(
            self._h, n, _ptr(seqs.offsets), _ptr(seqs.tau), _ptr(seqs.flavor), _ptr(seqs.dagger), float(t_obs),
            _ptr(op), _ptr(sign), _ptr(la), _ptr(st), int(nthreads))
        if st.any():
            raise ValueError(f"oracle rejected {int((st != 0).sum())} sequences")
        return sign.astype(np.int8), la

    def trace_obs(self, seqs: "SeqBatch", t_obs: float, obs: np.ndarray, nthreads: int = 0):
        """Traces with a diagonal operator inserted at t_obs (after every operator with tau < t_obs).

        obs: [nobs, 4^n_orb] values of each operator on every bitstring. Returns
        (sign int8 [n, nobs], log|T_O| float64 [n, nobs]).
        """
        obs = np.ascontiguousarray(obs, dtype=np.float64).reshape(-1, self.nstates)
        n, k = seqs.n, obs.shape[0]
        if k < 1:
            raise ValueError("at least one observable")
        sign = np.zeros((n, k), dtype=np.int32)
        la = np.zeros((n, k), dtype=np.float64)
        st = np.zeros(n, dtype=np.int32)
        self.threads_used = getattr(_lib, self.prefix + "trace_obs_batch")(
            self._h, n, _ptr(seqs.offsets), _ptr(seqs.tau), _ptr(seqs.flavor), _ptr(seqs.dagger), float(t_obs), k,
            _ptr(obs), _ptr(sign), _ptr(la), _ptr(st), int(nthreads))
        if st.any():
            raise ValueError(f"oracle rejected {int((st != 0).sum())} sequences (first at {int(np.argmax(st != 0))})")
        return sign.astype(np.int8), la


def spin_squared(n_orb: int) -> np.ndarray:
    """Total spin S^2 = S_x^2 + S_y^2 + S_z^2 over all bitstrings (dense), from
    S_+ = sum_a c^+_{a up} c_{a dn}, S_x = (S_+ + S_-)/2, S_y = (S_+ - S_-)/(2i),
    S_z = (N_up - N_dn)/2, with c_f built as Kronecker products carrying the
    Jordan-Wigner string of the lower flavors."""
    nf = 2 * n_orb
    a = np.array([[0.0, 1.0], [0.0, 0.0]])   # |1> -> |0> on one flavor
    Z = np.diag([1.0, -1.0])
    I2 = np.eye(2)
    c = []
    for f in range(nf):
        m = np.array([[1.0]])
        for g in reversed(range(nf)):        # most significant flavor first
            m = np.kron(m, a if g == f else (Z if g < f else I2))
        c.append(m)
    Sp = sum(c[2 * q].T @ c[2 * q + 1] for q in range(n_orb))
    Sm = Sp.T
    Sz = 0.5 * sum(c[2 * q].T @ c[2 * q] - c[2 * q + 1].T @ c[2 * q + 1] for q in range(n_orb))
    Sx, Sy2 = 0.5 * (Sp + Sm), -0.25 * (Sp - Sm) @ (Sp - Sm)
    return Sx @ Sx + Sy2 + Sz @ Sz


def observable_table(n_orb: int) -> np.ndarray:
    """Diagonal observables of the occupation basis, one row per operator, one column per
    bitstring x (bit f = n_f): n_f for f = 2a + s, then n_{a up} n_{a dn} per orbital a,
    then the projector on each (n_up, n_dn) sector, index n_up (n_orb + 1) + n_dn."""
    nf, ns = 2 * n_orb, 4 ** n_orb
    x = np.arange(ns)
    rows = [((x >> f) & 1).astype(np.float64) for f in range(nf)]
    rows += [(((x >> (2 * a)) & 1) * ((x >> (2 * a + 1)) & 1)).astype(np.float64) for a in range(n_orb)]
    nup = sum((x >> (2 * a)) & 1 for a in range(n_orb))
    ndn = sum((x >> (2 * a + 1)) & 1 for a in range(n_orb))
    for u in range(n_orb + 1):
        for d in range(n_orb + 1):
            rows.append(((nup == u) & (ndn == d)).astype(np.float64))
    return np.array(rows)


def measure(model: Model, seqs: "SeqBatch", nthreads: int = 0, spin: bool | None = None):
    """<O(beta/2)> = T_O / T per sequence for n_f, n_{a up} n_{a dn}, S^2 (when spin; by
    default for up to five orbitals, where the dense S^2 is small) and the (n_up, n_dn)
    projectors, in that order.

    Returns (obs [n, nobs] with NaN where T = 0, sign_T, log|T|)."""
    n = model.p.n_orb
    s, la, _ = model.trace(seqs, nthreads)
    tab = observable_table(n)
    so, lo = model.trace_obs(seqs, 0.5 * model.p.beta, tab, nthreads)
    with np.errstate(invalid="ignore", over="ignore"):
        val = so.astype(np.float64) * s[:, None].astype(np.float64) * np.exp(lo - la[:, None])
    spin = (n <= 5) if spin is None else spin
    col = np.full(seqs.n, np.nan)
    if spin:
        ss, ls = model.trace_op(seqs, 0.5 * model.p.beta, spin_squared(n), nthreads)
        with np.errstate(invalid="ignore", over="ignore"):
            col = ss.astype(np.float64) * s.astype(np.float64) * np.exp(ls - la)
    val = np.concatenate([val[:, :3 * n], col[:, None], val[:, 3 * n:]], axis=1)
    val[s == 0, :] = np.nan
    return val, s, la


@dataclass
class SeqBatch:
    """Sequences in CSR layout: ops of sequence i are offsets[i]..offsets[i+1]-1."""
    offsets: np.ndarray  # int32 [n+1]
    tau: np.ndarray      # float64 [K_total]
    flavor: np.ndarray   # uint8
    dagger: np.ndarray   # uint8

    def __post_init__(self):
        self.offsets = np.ascontiguousarray(self.offsets, dtype=np.int32)
        self.tau = np.ascontiguousarray(self.tau, dtype=np.float64)
        self.flavor = np.ascontiguousarray(self.flavor, dtype=np.uint8)
        self.dagger = np.ascontiguousarray(self.dagger, dtype=np.uint8)

    @property
    def n(self) -> int:
        return len(self.offsets) - 1

    def get(self, i: int):
        a, b = int(self.offsets[i]), int(self.offsets[i + 1])
        return list(zip(self.tau[a:b].tolist(), self.flavor[a:b].tolist(), self.dagger[a:b].tolist()))

    @staticmethod
    def from_lists(lists) -> "SeqBatch":
        offs = [0]
        tau, fl, dg = [], [], []
        for ops in lists:
            for t, f, d in ops:
                tau.append(t); fl.append(f); dg.append(d)
            offs.append(len(tau))
        return SeqBatch(np.array(offs), np.array(tau, dtype=np.float64), np.array(fl), np.array(dg))


def edit(ops, kind: int, flavor: int, t_dag: float, t_ann: float, rem_idx: int):
    """Apply one local update to a time-ordered operator list (Sec. II, local updates).

    kind 0 (insert): c^+_flavor at t_dag and c_flavor at t_ann, each placed after
    every existing operator at an equal time; if t_dag == t_ann the c goes first.
    kind 1 (remove): drop the operator at index rem_idx and the next operator of
    the same flavor after it in cyclic order, which must be of the other type (a
    c^+ with the c that closes its segment, or a c with the c^+ that closes its
    anti-segment).
    Returns the new list, or None if the move is malformed.
    """
    ops = list(ops)
    if kind == 0:
        new = [(t_ann, flavor, 0), (t_dag, flavor, 1)]
        if t_dag < t_ann:
            new = [(t_dag, flavor, 1), (t_ann, flavor, 0)]
        for t, f, d in new:
            pos = 0
            while pos < len(ops) and ops[pos][0] <= t:
                pos += 1
            ops.insert(pos, (t, f, d))
        return ops
    if kind == 1:
        K = len(ops)
        if not (0 <= rem_idx < K) or ops[rem_idx][1] != flavor:
            return None
        j = None
        for step in range(1, K):
            c = (rem_idx + step) % K
            if ops[c][1] == flavor:
                j = c
                break
        if j is None or ops[j][2] == ops[rem_idx][2]:
            return None
        return [op for i, op in enumerate(ops) if i not in (rem_idx, j)]
    return None


def ratio(model: Model, cur: SeqBatch, cur_sign, cur_logabs, moves, nthreads: int = 0):
    """Trace ratio of each proposed move against the given current (sign, log|T|).

    Returns (sign, logratio, new_sign, new_logabs). Walkers whose current sign is 0
    get sign 0 and logratio NaN.
    """
    lists = []
    for i in range(cur.n):
        e = edit(cur.get(i), int(moves["kind"][i]), int(moves["flavor"][i]), float(moves["t_dag"][i]),
                 float(moves["t_ann"][i]), int(moves["rem_idx"][i]))
        if e is None:
            raise ValueError(f"malformed move for walker {i}")
        lists.append(e)
    new = SeqBatch.from_lists(lists)
    ns, nl, _ = model.trace(new, nthreads)
    cs = np.asarray(cur_sign).astype(np.int64)
    sign = (ns.astype(np.int64) * cs).astype(np.int8)
    with np.errstate(invalid="ignore"):
        lr = np.where(ns != 0, nl - np.asarray(cur_logabs), -np.inf)
    lr = np.where(cs == 0, np.nan, lr)
    return sign, lr, ns, nl


def classify(sign64, lt64, signx, ltx, rel: float = 1e-8):
    """Conditioning class of each trace: 0 structural zero, 1 numerical zero, 2 regular.

    Structural zero: the FP64 oracle returns exactly zero (no contributing path).
    Numerical zero: FP64 and the long-double twin disagree by more than ``rel``
    relative (or in sign), which happens when the exact value vanishes by a
    symmetry the (n_up, n_dn) sectors do not resolve and both results are rounding
    noise. Regular: everything else.
    """
    sign64 = np.asarray(sign64); signx = np.asarray(signx)
    out = np.full(len(sign64), 2, dtype=np.int8)
    for i in range(len(sign64)):
        if sign64[i] == 0 and signx[i] == 0:
            out[i] = 0
        elif sign64[i] != signx[i] or not (abs(math.expm1(float(lt64[i]) - float(ltx[i]))) <= rel):
            out[i] = 1
    return out
