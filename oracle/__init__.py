"""CPU oracle of the VBDR method (arXiv 1810.13132) -- TEST INFRASTRUCTURE.

Only ``tests/``, ``__graft_entry__.smoke()`` and the CPU-baseline leg of
``bench.py`` may import this package.  It shares no code with the CUDA
library in ``paper_1810_13132_gb300/``: the oracle is plain single-threaded C
(``vbdr_oracle.c``) plus the exact ground truth of Definition 1 written with
numpy set operations (``exact.py``).

Functions and what they follow:

* ``Oracle.scan``      -- Alg. 4 (serial), Alg. 7 (gfast), Alg. 9 (gsmall)
* ``Oracle.slide``     -- Alg. 1 / Alg. 6 then Alg. 2 (serial, gfast);
                          Alg. 2 then Alg. 8 (gsmall)
* ``Oracle.estimate``  -- Alg. 3 + Alg. 5 + the vHLL estimator (Sec. 4.1)
* ``exact.window_cardinalities`` -- Definition 1, |OP(aip, t, k)|
"""
from __future__ import annotations

import ctypes
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "vbdr_oracle.c")
_LIB_PATH = os.path.join(_HERE, "libvbdr_oracle.so")

GFAST, GSMALL, SERIAL = 0, 1, 2
VARIANTS = {"gfast": GFAST, "gsmall": GSMALL, "serial": SERIAL}


def build(force: bool = False) -> str:
    """Compile the oracle with gcc (-O2, plain C11).  Returns the .so path."""
    if (not force and os.path.exists(_LIB_PATH)
            and os.path.getmtime(_LIB_PATH) >= os.path.getmtime(_SRC)):
        return _LIB_PATH
    tmp = _LIB_PATH + f".tmp{os.getpid()}"
    subprocess.check_call(["gcc", "-std=c11", "-O2", "-fPIC", "-shared",
                           "-fno-fast-math", "-o", tmp, _SRC, "-lm"])
    os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


_lib = None


def lib() -> ctypes.CDLL:
    global _lib
    if _lib is None:
        # ORACLE_LIB_OVERRIDE lets the mutation test load a deliberately
        # broken build of this same source, to show the pins catch it.
        L = ctypes.CDLL(os.environ.get("ORACLE_LIB_OVERRIDE") or build())
        u8p = ctypes.POINTER(ctypes.c_uint8)
        u32p = ctypes.POINTER(ctypes.c_uint32)
        u64p = ctypes.POINTER(ctypes.c_uint64)
        f64p = ctypes.POINTER(ctypes.c_double)
        L.orc_mix64.restype = ctypes.c_uint64
        L.orc_mix64.argtypes = [ctypes.c_uint64]
        L.orc_splitmix64_next.restype = ctypes.c_uint64
        L.orc_splitmix64_next.argtypes = [u64p]
        L.orc_H.restype = ctypes.c_uint64
        L.orc_H.argtypes = [ctypes.c_uint64] * 3
        L.orc_create.restype = ctypes.c_void_p
        L.orc_create.argtypes = [ctypes.c_int, ctypes.c_uint32, ctypes.c_uint64,
                                 ctypes.c_uint32, ctypes.c_uint32,
                                 ctypes.c_uint32, ctypes.c_uint64]
        L.orc_destroy.argtypes = [ctypes.c_void_p]
        for name in ("orc_dr_max", "orc_R"):
            getattr(L, name).restype = ctypes.c_uint32
            getattr(L, name).argtypes = [ctypes.c_void_p]
        L.orc_A1.restype = ctypes.c_uint64
        L.orc_A1.argtypes = [ctypes.c_void_p]
        L.orc_host_b.restype = ctypes.c_uint32
        L.orc_host_b.argtypes = [ctypes.c_void_p, ctypes.c_uint32]
        L.orc_get_phy_idx.restype = ctypes.c_uint64
        L.orc_get_phy_idx.argtypes = [ctypes.c_void_p, ctypes.c_uint32,
                                      ctypes.c_uint32]
        L.orc_hash_pair.argtypes = [ctypes.c_void_p, ctypes.c_uint32,
                                    ctypes.c_uint32, u64p, u32p, u32p]
        L.orc_scan.argtypes = [ctypes.c_void_p, u32p, ctypes.c_uint64]
        L.orc_slide.argtypes = [ctypes.c_void_p]
        L.orc_estimate.restype = ctypes.c_int
        L.orc_estimate.argtypes = [ctypes.c_void_p, u32p, ctypes.c_uint64, f64p]
        L.orc_host_registers.argtypes = [ctypes.c_void_p, ctypes.c_uint32,
                                         u64p, u64p, u64p, u32p]
        L.orc_get_state.argtypes = [ctypes.c_void_p, u8p, u32p, u8p, u8p]
        L.orc_set_registers.argtypes = [ctypes.c_void_p, u8p]
        L.orc_set_state.argtypes = [ctypes.c_void_p, u8p, u32p]
        L.orc_pool_sums_get.argtypes = [ctypes.c_void_p, u64p, u64p]
        L.orc_features.restype = ctypes.c_int
        L.orc_features.argtypes = [ctypes.c_void_p, u32p, ctypes.c_uint64, f64p, f64p]
        L.orc_load_virtual_registers.argtypes = [ctypes.c_void_p, u32p, u64p,
                                                 ctypes.c_uint64, u8p]
        L.orc_hll_alpha.restype = ctypes.c_double
        L.orc_hll_alpha.argtypes = [ctypes.c_double]
        L.orc_hll.restype = ctypes.c_double
        L.orc_hll.argtypes = [ctypes.c_double, ctypes.c_uint64, ctypes.c_uint64]
        L.orc_vhll.restype = ctypes.c_double
        L.orc_vhll.argtypes = [ctypes.c_double, ctypes.c_double,
                               ctypes.c_uint64, ctypes.c_uint64,
                               ctypes.c_uint64, ctypes.c_uint64]
        L.orc_loglog_alpha.restype = ctypes.c_double
        L.orc_loglog_alpha.argtypes = [ctypes.c_double]
        L.orc_loglog.restype = ctypes.c_double
        L.orc_loglog.argtypes = [ctypes.c_double, ctypes.c_uint64]
        L.orc_pcsa.restype = ctypes.c_double
        L.orc_pcsa.argtypes = [ctypes.c_double, ctypes.c_uint64]
        L.orc_estimate_alt.restype = ctypes.c_int
        L.orc_estimate_alt.argtypes = [ctypes.c_void_p, ctypes.c_int, u32p, ctypes.c_uint64,
                                       f64p]
        L.orc_pool_sums_alt.argtypes = [ctypes.c_void_p, u64p, u64p]
        L.orc_get_pcsa.argtypes = [ctypes.c_void_p, u8p]
        L.orc_table1_bits.restype = ctypes.c_uint32
        L.orc_table1_bits.argtypes = [ctypes.c_void_p, ctypes.c_int]
        _lib = L
    return _lib


def _ptr(a: np.ndarray, ctype):
    return a.ctypes.data_as(ctypes.POINTER(ctype))


def mix64(x: int) -> int:
    return lib().orc_mix64(x)


def H(x: int, N: int, A: int) -> int:
    return lib().orc_H(x, N, A)


def splitmix64_sequence(seed: int, n: int) -> list[int]:
    st = ctypes.c_uint64(seed)
    return [lib().orc_splitmix64_next(ctypes.byref(st)) for _ in range(n)]


def hll(m: float, S: int, V: int) -> float:
    return lib().orc_hll(float(m), int(S), int(V))


def hll_alpha(m: float) -> float:
    return lib().orc_hll_alpha(float(m))


def vhll(Z: float, g: float, S: int, V: int, S_Z: int, V_Z: int) -> float:
    return lib().orc_vhll(float(Z), float(g), int(S), int(V), int(S_Z), int(V_Z))


def loglog_alpha(m: float) -> float:
    return lib().orc_loglog_alpha(float(m))


def loglog(m: float, L: int) -> float:
    return lib().orc_loglog(float(m), int(L))


def pcsa(m: float, P: int) -> float:
    return lib().orc_pcsa(float(m), int(P))


ESTIMATORS = {"loglog": 1, "pcsa": 2}


class Oracle:
    """One VBDR instance with logical (unpacked) state.

    ``variant`` is "gfast" (Alg. 6/7), "gsmall" (Alg. 8/9) or "serial"
    (Alg. 1/4).  ``b`` is log2 g of every host; ``group_rule=1`` gives four
    mixed groups ``b_min .. b_min+3``.
    """

    def __init__(self, variant: str, k: int, Z: int, b: int, seed: int,
                 b_min: int | None = None, group_rule: int = 0):
        self.variant = variant
        self.k, self.Z, self.b, self.seed = k, Z, b, seed
        self.b_min = b if b_min is None else b_min
        self.group_rule = group_rule
        self._h = lib().orc_create(VARIANTS[variant], k, Z, b, self.b_min,
                                   group_rule, seed)
        if not self._h:
            raise ValueError("invalid oracle parameters")
        self.R = lib().orc_R(self._h)
        self.dr_max = lib().orc_dr_max(self._h)

    def __del__(self):
        h = getattr(self, "_h", None)
        if h:
            lib().orc_destroy(h)
            self._h = None

    # -- hashing -----------------------------------------------------------
    def host_b(self, aip: int) -> int:
        return lib().orc_host_b(self._h, aip)

    def phy_idx(self, aip: int, i: int) -> int:
        return lib().orc_get_phy_idx(self._h, aip, i)

    def hash_pair(self, aip: int, bip: int) -> tuple[int, int, int]:
        """(pidx, rho, vidx) of one pair."""
        p = ctypes.c_uint64()
        r = ctypes.c_uint32()
        v = ctypes.c_uint32()
        lib().orc_hash_pair(self._h, aip, bip, ctypes.byref(p),
                            ctypes.byref(r), ctypes.byref(v))
        return p.value, r.value, v.value

    # -- the method ----------------------------------------------------------
    def scan(self, pairs: np.ndarray) -> None:
        pairs = np.ascontiguousarray(pairs, dtype=np.uint32).reshape(-1, 2)
        lib().orc_scan(self._h, _ptr(pairs, ctypes.c_uint32), pairs.shape[0])

    def slide(self) -> None:
        lib().orc_slide(self._h)

    def estimate(self, aips: np.ndarray) -> np.ndarray:
        aips = np.ascontiguousarray(aips, dtype=np.uint32)
        out = np.empty(aips.shape[0], dtype=np.float64)
        rc = lib().orc_estimate(self._h, _ptr(aips, ctypes.c_uint32),
                                aips.shape[0], _ptr(out, ctypes.c_double))
        if rc != 0:
            raise RuntimeError("estimate before the first slide")
        return out

    def estimate_alt(self, aips: np.ndarray, estimator: str) -> np.ndarray:
        """LogLog ("loglog") or PCSA ("pcsa", gsmall only) estimates."""
        aips = np.ascontiguousarray(aips, dtype=np.uint32)
        out = np.empty(aips.shape[0], dtype=np.float64)
        rc = lib().orc_estimate_alt(self._h, ESTIMATORS[estimator], _ptr(aips, ctypes.c_uint32),
                                    aips.shape[0], _ptr(out, ctypes.c_double))
        if rc == -1:
            raise RuntimeError("estimate before the first slide")
        if rc == -2:
            raise ValueError("PCSA needs the gsmall layout")
        return out

    def pcsa_statistics(self) -> np.ndarray:
        out = np.empty(self.Z, dtype=np.uint8)
        lib().orc_get_pcsa(self._h, _ptr(out, ctypes.c_uint8))
        return out

    def pool_sums_alt(self) -> tuple[int, int]:
        """(sum of registers, sum of PCSA statistics) over the pool."""
        L, P = ctypes.c_uint64(), ctypes.c_uint64()
        lib().orc_pool_sums_alt(self._h, ctypes.byref(L), ctypes.byref(P))
        return L.value, P.value

    def features(self, aips: np.ndarray):
        """(X [n, 80] float64, n_plain [n]) of the learned correction."""
        aips = np.ascontiguousarray(aips, dtype=np.uint32)
        X = np.empty((aips.size, 80), dtype=np.float64)
        est = np.empty(aips.size, dtype=np.float64)
        rc = lib().orc_features(self._h, _ptr(aips, ctypes.c_uint32), aips.size,
                                _ptr(X, ctypes.c_double), _ptr(est, ctypes.c_double))
        if rc != 0:
            raise RuntimeError("features before the first slide")
        return X, est

    def host_registers(self, aip: int):
        """(S, V, sum_lbp1, hist64) of one host's virtual registers."""
        S, V, L = ctypes.c_uint64(), ctypes.c_uint64(), ctypes.c_uint64()
        hist = np.zeros(64, dtype=np.uint32)
        lib().orc_host_registers(self._h, aip, ctypes.byref(S), ctypes.byref(V),
                                 ctypes.byref(L), _ptr(hist, ctypes.c_uint32))
        return S.value, V.value, L.value, hist

    # -- inspection ----------------------------------------------------------
    def state(self) -> dict:
        dr = np.empty((self.Z, self.R), dtype=np.uint8)
        bs = np.empty(self.Z, dtype=np.uint32)
        reg = np.empty(self.Z, dtype=np.uint8)
        now = np.empty(self.Z, dtype=np.uint8)
        lib().orc_get_state(self._h, _ptr(dr, ctypes.c_uint8),
                            _ptr(bs, ctypes.c_uint32), _ptr(reg, ctypes.c_uint8),
                            _ptr(now, ctypes.c_uint8))
        return {"dr": dr, "bs": bs, "reg": reg, "now": now}

    def registers(self) -> np.ndarray:
        reg = np.empty(self.Z, dtype=np.uint8)
        lib().orc_get_state(self._h, None, None, _ptr(reg, ctypes.c_uint8), None)
        return reg

    def set_state(self, dr: np.ndarray | None = None, bs: np.ndarray | None = None) -> None:
        d = None if dr is None else np.ascontiguousarray(dr, dtype=np.uint8)
        b = None if bs is None else np.ascontiguousarray(bs, dtype=np.uint32)
        lib().orc_set_state(self._h, None if d is None else _ptr(d, ctypes.c_uint8),
                            None if b is None else _ptr(b, ctypes.c_uint32))

    def set_registers(self, reg: np.ndarray) -> None:
        reg = np.ascontiguousarray(reg, dtype=np.uint8)
        assert reg.shape == (self.Z,)
        lib().orc_set_registers(self._h, _ptr(reg, ctypes.c_uint8))

    def load_virtual_registers(self, aips: np.ndarray, offsets: np.ndarray,
                               vregs: np.ndarray) -> None:
        aips = np.ascontiguousarray(aips, dtype=np.uint32)
        offsets = np.ascontiguousarray(offsets, dtype=np.uint64)
        vregs = np.ascontiguousarray(vregs, dtype=np.uint8)
        lib().orc_load_virtual_registers(self._h, _ptr(aips, ctypes.c_uint32),
                                         _ptr(offsets, ctypes.c_uint64), aips.size,
                                         _ptr(vregs, ctypes.c_uint8))

    def pool_sums(self) -> tuple[int, int]:
        S, V = ctypes.c_uint64(), ctypes.c_uint64()
        lib().orc_pool_sums_get(self._h, ctypes.byref(S), ctypes.byref(V))
        return S.value, V.value

    def table1_bits(self, variant: str) -> int:
        return lib().orc_table1_bits(self._h, VARIANTS[variant])
