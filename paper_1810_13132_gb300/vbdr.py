"""Python binding of the VBDR C ABI (include/vbdr.h) -- argument marshalling only.

Every step of the method runs in the CUDA library libvbdr.so; this module only
passes device pointers (``torch.Tensor.data_ptr()``) and the current CUDA
stream.  There is no CPU fallback: without the library or a GPU every call
raises.
"""
from __future__ import annotations

import ctypes
import os
from dataclasses import dataclass

import numpy as np

from . import _build

VBDR_GFAST, VBDR_GSMALL, VBDR_SERIAL = 0, 1, 2
LAYOUTS = {"gfast": VBDR_GFAST, "gsmall": VBDR_GSMALL, "serial": VBDR_SERIAL}

STATUS = {0: "VBDR_OK", -1: "VBDR_EINVAL", -2: "VBDR_ENOMEM", -3: "VBDR_ECUDA",
          -4: "VBDR_ERANGE", -5: "VBDR_EORDER", -6: "VBDR_ETIMEOUT"}


class VbdrError(RuntimeError):
    def __init__(self, fn: str, code: int):
        self.code = code
        super().__init__(f"{fn} failed: {STATUS.get(code, code)} ({_strerror(code)})")


class vbdr_config(ctypes.Structure):
    _fields_ = [("k", ctypes.c_uint32), ("log2_g", ctypes.c_uint32),
                ("log2_g_min", ctypes.c_uint32), ("group_rule", ctypes.c_uint32),
                ("layout", ctypes.c_uint32), ("reserved", ctypes.c_uint32),
                ("num_bdr", ctypes.c_uint64), ("seed", ctypes.c_uint64)]


# Every symbol include/vbdr.h declares, with (restype, argtypes).
_VP, _U32, _U64 = ctypes.c_void_p, ctypes.c_uint32, ctypes.c_uint64
_SIGS = {
    "vbdr_create": (ctypes.c_int, [ctypes.POINTER(vbdr_config), ctypes.POINTER(_VP)]),
    "vbdr_destroy": (ctypes.c_int, [_VP]),
    "vbdr_scan_slice": (ctypes.c_int, [_VP, _VP, _U64, _VP]),
    "vbdr_scan_slice_host": (ctypes.c_int, [_VP, _VP, _U64, _VP]),
    "vbdr_slide": (ctypes.c_int, [_VP, _VP]),
    "vbdr_estimate": (ctypes.c_int, [_VP, _VP, _U64, _VP, _VP]),
    "vbdr_estimate_host": (ctypes.c_int, [_VP, _VP, _U64, _VP, _VP]),
    "vbdr_estimate_alt": (ctypes.c_int, [_VP, _VP, _U64, _VP, ctypes.c_int, _VP]),
    "vbdr_copy_pool_sums_alt": (ctypes.c_int, [_VP, ctypes.POINTER(_U64), ctypes.POINTER(_U64),
                                               _VP]),
    "vbdr_copy_pcsa": (ctypes.c_int, [_VP, _VP, _VP]),
    "vbdr_selftest_bounded_wait": (ctypes.c_int, [_U32, _VP]),
    "vbdr_check_flags": (ctypes.c_int, [_VP, ctypes.POINTER(_U32), ctypes.POINTER(ctypes.c_int)]),
    "vbdr_plan_create": (ctypes.c_int, [_VP, _VP, _U64, ctypes.POINTER(_VP), _VP]),
    "vbdr_plan_destroy": (ctypes.c_int, [_VP]),
    "vbdr_plan_create_learned": (ctypes.c_int, [_VP, _VP, _U64, ctypes.POINTER(_VP), _VP]),
    "vbdr_estimate_learned_planned": (ctypes.c_int, [_VP, _VP, _VP, _VP, _VP]),
    "vbdr_plan_info": (ctypes.c_int, [_VP, ctypes.POINTER(_U64), ctypes.POINTER(_U64),
                                      ctypes.POINTER(_U64)]),
    "vbdr_plan_status": (ctypes.c_int, [_VP]),
    "vbdr_estimate_planned": (ctypes.c_int, [_VP, _VP, _VP, _VP]),
    "vbdr_estimate_planned_compact": (ctypes.c_int, [_VP, _VP, _VP, ctypes.c_float, _VP, _VP]),
    "vbdr_estimate_planned_host": (ctypes.c_int, [_VP, _VP, _VP, _VP]),
    "vbdr_get_dims": (ctypes.c_int, [_VP, ctypes.POINTER(_U32), ctypes.POINTER(_U32),
                                     ctypes.POINTER(_U32)]),
    "vbdr_copy_state": (ctypes.c_int, [_VP, _VP, _VP, _VP, _VP]),
    "vbdr_copy_pool_sums": (ctypes.c_int, [_VP, ctypes.POINTER(_U64),
                                           ctypes.POINTER(_U64), _VP]),
    "vbdr_strerror": (ctypes.c_char_p, [ctypes.c_int]),
    "vbdr_load_virtual_registers": (ctypes.c_int, [_VP, _VP, _VP, _U64, _VP, _VP]),
    "vbdr_set_estimate_launch": (ctypes.c_int, [_VP, _U32, _U32]),
    "vbdr_autotune_estimate": (ctypes.c_int, [_VP, _VP, _U64, _VP, ctypes.POINTER(_U32),
                                              ctypes.POINTER(_U32), _VP]),
    "vbdr_mlp_num_params": (ctypes.c_int, []),
    "vbdr_mlp_create": (ctypes.c_int, [_U64, ctypes.POINTER(_VP)]),
    "vbdr_mlp_destroy": (ctypes.c_int, [_VP]),
    "vbdr_mlp_set_params": (ctypes.c_int, [_VP, _VP, ctypes.c_float]),
    "vbdr_mlp_get_params": (ctypes.c_int, [_VP, _VP, ctypes.POINTER(ctypes.c_float)]),
    "vbdr_mlp_train": (ctypes.c_int, [_VP, _VP, _VP, _U64, _U32, _U32, ctypes.c_float,
                                      ctypes.c_float, _U64, _VP, _VP]),
    "vbdr_mlp_gradient": (ctypes.c_int, [_VP, _VP, _VP, _U64, _VP,
                                         ctypes.POINTER(ctypes.c_float), _VP]),
    "vbdr_mlp_forward": (ctypes.c_int, [_VP, _VP, _U64, _VP, _VP]),
    "vbdr_features": (ctypes.c_int, [_VP, _VP, _U64, _VP, _VP, _VP]),
    "vbdr_estimate_learned": (ctypes.c_int, [_VP, _VP, _VP, _U64, _VP, _VP]),
    "vbdr_scan_slice_devn": (ctypes.c_int, [_VP, _VP, _VP, _U64, _VP]),
    "vbdr_server_create": (ctypes.c_int, [ctypes.c_void_p, ctypes.POINTER(_VP)]),
    "vbdr_server_destroy": (ctypes.c_int, [_VP]),
    "vbdr_server_tenant_bytes": (_U64, [ctypes.POINTER(vbdr_config), _U64, _U64]),
    "vbdr_server_open": (ctypes.c_int, [_VP, ctypes.POINTER(vbdr_config), _U64, _VP, _U64, _VP,
                                        _U32, ctypes.POINTER(_U32)]),
    "vbdr_server_close": (ctypes.c_int, [_VP, _U32]),
    "vbdr_server_submit": (ctypes.c_int, [_VP, _U32, _VP, _U64, ctypes.POINTER(_U64)]),
    "vbdr_server_wait": (ctypes.c_int, [_VP, _U32, _U64, _VP, _U32,
                                        ctypes.POINTER(ctypes.c_float),
                                        ctypes.POINTER(ctypes.c_float)]),
    "vbdr_server_in_use": (ctypes.c_int, [_VP, ctypes.POINTER(_U64), ctypes.POINTER(_U32)]),
    "vbdr_server_tenant_handle": (ctypes.c_int, [_VP, _U32, ctypes.POINTER(_VP)]),
    "vbdr_state_bytes": (ctypes.c_int, [_VP, ctypes.POINTER(_U64)]),
    "vbdr_save": (ctypes.c_int, [_VP, _VP, _U64, _VP]),
    "vbdr_load": (ctypes.c_int, [_VP, _VP, _U64, _VP]),
    "vbdr_set_scan_mode": (ctypes.c_int, [_VP, ctypes.c_int]),
    "vbdr_state_pointers": (ctypes.c_int, [_VP, ctypes.POINTER(_VP), ctypes.POINTER(_U64),
                                           ctypes.POINTER(_VP), ctypes.POINTER(_VP)]),
    "vbdr_route_records": (ctypes.c_int, [_VP, _VP, _U64, _U32, _VP, _U64, _VP, _VP]),
    "vbdr_apply_records": (ctypes.c_int, [_VP, _VP, _U64, _VP]),
    "vbdr_merge_slice_state": (ctypes.c_int, [_VP, _VP, _VP]),
    "vbdr_set_registers": (ctypes.c_int, [_VP, _VP, _VP, _VP]),
    "vbdr_estimate_registers_noalloc": (ctypes.c_int, [_VP, _U64, _U32, _U64, _VP, _U64, _VP,
                                                       _VP]),
}

_lib = None


def _checked() -> bool:
    # VBDR_CHECKED=1 selects the bounds-checked build (libvbdr_check.so)
    return os.environ.get("VBDR_CHECKED", "") == "1"


def library_path() -> str:
    return _build.LIB_CHECK if _checked() else _build.LIB


def load(build_if_missing: bool = True) -> ctypes.CDLL:
    """Load libvbdr.so, or libvbdr_check.so when VBDR_CHECKED=1 (building
    it with nvcc first if it is missing)."""
    global _lib
    if _lib is None:
        path = _build.build(check=_checked()) if build_if_missing else library_path()
        if not os.path.exists(path):
            raise RuntimeError(f"CUDA library missing: {path}")
        L = ctypes.CDLL(path)
        for name, (res, args) in _SIGS.items():
            fn = getattr(L, name)
            fn.restype = res
            fn.argtypes = args
        _lib = L
    return _lib


def exported_symbols() -> list[str]:
    return sorted(_SIGS)


def _strerror(code: int) -> str:
    try:
        return load(build_if_missing=False).vbdr_strerror(code).decode()
    except Exception:
        return "?"


def _check(fn: str, rc: int) -> None:
    if rc != 0:
        raise VbdrError(fn, rc)


def _stream_ptr(stream=None) -> int:
    import torch
    s = stream if stream is not None else torch.cuda.current_stream()
    return int(s.cuda_stream)


ESTIMATORS = {"hll": 0, "loglog": 1, "pcsa": 2}


@dataclass
class Config:
    k: int
    num_bdr: int
    log2_g: int
    seed: int = 0x9E3779B97F4A7C15
    layout: str = "gfast"
    log2_g_min: int = 0
    group_rule: int = 0

    def to_c(self) -> vbdr_config:
        return vbdr_config(self.k, self.log2_g, self.log2_g_min, self.group_rule,
                           LAYOUTS[self.layout], 0, self.num_bdr, self.seed)


class Vbdr:
    """One VBDR instance with device-resident state (see include/vbdr.h).

    ``scan(pairs)`` takes an (n, 2) uint32/int32 CUDA tensor of (aip, bip),
    ``slide()`` closes the slice, ``estimate(aips)`` returns float32
    estimates on the device.  Calls run on the current torch CUDA stream.
    """

    def __init__(self, cfg: Config, _borrowed=None):
        import torch
        if not torch.cuda.is_available():
            raise RuntimeError("VBDR needs a CUDA GPU; no CPU fallback exists")
        torch.cuda.init()
        self.cfg = cfg
        self._L = load()
        self._owned = _borrowed is None
        if _borrowed is None:
            h = ctypes.c_void_p()
            c = cfg.to_c()
            _check("vbdr_create", self._L.vbdr_create(ctypes.byref(c), ctypes.byref(h)))
        else:
            h = _borrowed
        self._h = h
        R, w, P = ctypes.c_uint32(), ctypes.c_uint32(), ctypes.c_uint32()
        _check("vbdr_get_dims", self._L.vbdr_get_dims(h, ctypes.byref(R), ctypes.byref(w),
                                                      ctypes.byref(P)))
        self.R, self.w, self.words = R.value, w.value, P.value

    def close(self) -> None:
        if getattr(self, "_h", None):
            if self._owned:
                self._L.vbdr_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    SCAN_MODES = {"direct": 0, "bucketed": 1}

    def set_scan_mode(self, mode: str) -> None:
        """"direct" (default) or "bucketed" scan kernels (same state)."""
        _check("vbdr_set_scan_mode", self._L.vbdr_set_scan_mode(self._h, self.SCAN_MODES[mode]))

    # -- the hot path ----------------------------------------------------------
    def scan(self, pairs, stream=None) -> None:
        import torch
        assert pairs.is_cuda and pairs.is_contiguous()
        assert pairs.dtype in (torch.int32, torch.uint32)
        n = pairs.numel() // 2
        _check("vbdr_scan_slice", self._L.vbdr_scan_slice(
            self._h, pairs.data_ptr() if n else None, n, _stream_ptr(stream)))

    def scan_host(self, pairs: np.ndarray, stream=None) -> None:
        """Scan pairs held in host memory (numpy or pinned torch CPU tensor)."""
        ptr, n = _host_ptr(pairs, 2)
        _check("vbdr_scan_slice_host", self._L.vbdr_scan_slice_host(
            self._h, ptr, n, _stream_ptr(stream)))

    def slide(self, stream=None) -> None:
        _check("vbdr_slide", self._L.vbdr_slide(self._h, _stream_ptr(stream)))

    def estimate(self, aips, out=None, stream=None, estimator: str = "hll"):
        """Estimates of aips; estimator "hll" (vHLL), "loglog" or "pcsa"
        (gsmall only), see include/vbdr.h."""
        import torch
        assert aips.is_cuda and aips.is_contiguous()
        n = aips.numel()
        if out is None:
            out = torch.empty(n, dtype=torch.float32, device=aips.device)
        if estimator == "hll":
            _check("vbdr_estimate", self._L.vbdr_estimate(
                self._h, aips.data_ptr() if n else None, n, out.data_ptr() if n else None,
                _stream_ptr(stream)))
        else:
            _check("vbdr_estimate_alt", self._L.vbdr_estimate_alt(
                self._h, aips.data_ptr() if n else None, n, out.data_ptr() if n else None,
                ESTIMATORS[estimator], _stream_ptr(stream)))
        return out

    def estimate_host(self, aips, out, stream=None) -> None:
        pa, n = _host_ptr(aips, 1)
        po, n2 = _host_ptr(out, 1)
        assert n == n2
        _check("vbdr_estimate_host", self._L.vbdr_estimate_host(
            self._h, pa, n, po, _stream_ptr(stream)))

    # -- planned estimation ----------------------------------------------------
    def plan(self, aips, stream=None, learned: bool = False) -> "Plan":
        """Estimate plan of a host list (int32/uint32 CUDA tensor); see Plan.
        learned=True builds the smaller-block plan the planned learned
        correction needs (it also serves estimate_planned)."""
        assert aips.is_cuda and aips.is_contiguous()
        n = aips.numel()
        p = ctypes.c_void_p()
        fn = "vbdr_plan_create_learned" if learned else "vbdr_plan_create"
        _check(fn, getattr(self._L, fn)(
            self._h, aips.data_ptr() if n else None, n, ctypes.byref(p), _stream_ptr(stream)))
        return Plan(self._L, p, n)

    def estimate_learned_planned(self, mlp: "Mlp", plan: "Plan", out=None, stream=None):
        """Corrected estimates of a learned plan's hosts (float32 CUDA tensor)."""
        import torch
        if out is None:
            out = torch.empty(plan.n_hosts, dtype=torch.float32, device="cuda")
        assert out.is_cuda and out.numel() >= plan.n_hosts
        _check("vbdr_estimate_learned_planned", self._L.vbdr_estimate_learned_planned(
            self._h, mlp._h, plan._p, out.data_ptr() if plan.n_hosts else None,
            _stream_ptr(stream)))
        return out

    def estimate_planned(self, plan: "Plan", out=None, stream=None):
        """Estimates of the plan's hosts (float32 CUDA tensor, plan order)."""
        import torch
        if out is None:
            out = torch.empty(plan.n_hosts, dtype=torch.float32, device="cuda")
        assert out.is_cuda and out.numel() >= plan.n_hosts
        _check("vbdr_estimate_planned", self._L.vbdr_estimate_planned(
            self._h, plan._p, out.data_ptr() if plan.n_hosts else None, _stream_ptr(stream)))
        return out

    def estimate_planned_compact(self, plan: "Plan", net: "CompactNet", out=None, stream=None):
        """Estimates of the plan's hosts with the compact learned correction
        applied in the same kernel (float32 CUDA tensor, plan order)."""
        import torch
        if out is None:
            out = torch.empty(plan.n_hosts, dtype=torch.float32, device="cuda")
        assert out.is_cuda and out.numel() >= plan.n_hosts
        _check("vbdr_estimate_planned_compact", self._L.vbdr_estimate_planned_compact(
            self._h, plan._p, net.theta.ctypes.data, net.nmax,
            out.data_ptr() if plan.n_hosts else None, _stream_ptr(stream)))
        return out

    def estimate_planned_host(self, plan: "Plan", out, stream=None) -> None:
        po, n = _host_ptr(out, 1)
        assert n >= plan.n_hosts
        _check("vbdr_estimate_planned_host", self._L.vbdr_estimate_planned_host(
            self._h, plan._p, po, _stream_ptr(stream)))

    # -- batched estimation --------------------------------------------------------
    def load_virtual_registers(self, aips, offsets, vregs, stream=None) -> None:
        """Register-level state (device tensors: int32 aips, int64 offsets,
        uint8 virtual registers, host-major)."""
        _check("vbdr_load_virtual_registers", self._L.vbdr_load_virtual_registers(
            self._h, aips.data_ptr(), offsets.data_ptr(), aips.numel(), vregs.data_ptr(),
            _stream_ptr(stream)))

    def set_estimate_launch(self, lanes: int, threads: int) -> None:
        _check("vbdr_set_estimate_launch", self._L.vbdr_set_estimate_launch(
            self._h, lanes, threads))

    def autotune_estimate(self, aips, out=None, stream=None) -> tuple[int, int]:
        import torch
        if out is None:
            out = torch.empty(aips.numel(), dtype=torch.float32, device=aips.device)
        lanes, threads = ctypes.c_uint32(), ctypes.c_uint32()
        _check("vbdr_autotune_estimate", self._L.vbdr_autotune_estimate(
            self._h, aips.data_ptr(), aips.numel(), out.data_ptr(), ctypes.byref(lanes),
            ctypes.byref(threads), _stream_ptr(stream)))
        return lanes.value, threads.value

    # -- learned correction ------------------------------------------------------
    def features(self, aips, stream=None):
        """(X bf16 [n, 48] live features, plain estimates f32 [n]) on the device."""
        import torch
        n = aips.numel()
        X = torch.empty((n, 48), dtype=torch.bfloat16, device=aips.device)
        plain = torch.empty(n, dtype=torch.float32, device=aips.device)
        _check("vbdr_features", self._L.vbdr_features(
            self._h, aips.data_ptr(), n, X.data_ptr(), plain.data_ptr(), _stream_ptr(stream)))
        return X, plain

    def estimate_learned(self, mlp: "Mlp", aips, out=None, stream=None):
        import torch
        n = aips.numel()
        if out is None:
            out = torch.empty(n, dtype=torch.float32, device=aips.device)
        _check("vbdr_estimate_learned", self._L.vbdr_estimate_learned(
            self._h, mlp._h, aips.data_ptr(), n, out.data_ptr(), _stream_ptr(stream)))
        return out

    # -- several GPUs ---------------------------------------------------------------
    def _pointers(self):
        st, w, reg, pc = _VP(), _U64(), _VP(), _VP()
        _check("vbdr_state_pointers", self._L.vbdr_state_pointers(
            self._h, ctypes.byref(st), ctypes.byref(w), ctypes.byref(reg), ctypes.byref(pc)))
        return st.value, w.value, reg.value, pc.value

    def slice_state(self, stream=None):
        """A copy (int32 CUDA tensor) of the slice state the replicas merge."""
        ptr, words, _, _ = self._pointers()
        return _device_copy(ptr, words, "<i4")

    def merge_slice_state(self, other, stream=None) -> None:
        """Merge another replica's slice state (int32 CUDA tensor laid out as
        slice_state() returns it) into this handle's."""
        ptr, words, _, _ = self._pointers()
        assert other.is_cuda and other.is_contiguous() and other.numel() == words
        assert other.dtype in (torch_int32(), torch_uint32())
        _check("vbdr_merge_slice_state", self._L.vbdr_merge_slice_state(
            self._h, other.data_ptr(), _stream_ptr(stream)))

    def route_records(self, pairs, n_ranks: int, cap: int | None = None, stream=None):
        """(records [n_ranks, cap] int32 CUDA tensor, fill [n_ranks] int64):
        the pairs hashed into records pidx << 5 | (LBP1 - 1), grouped by the
        rank owning pidx."""
        import torch
        assert pairs.is_cuda and pairs.is_contiguous()
        n = pairs.numel() // 2
        cap = n if cap is None else cap
        recs = torch.empty((n_ranks, max(cap, 1)), dtype=torch.int32, device="cuda")
        fill = torch.empty(n_ranks, dtype=torch.int64, device="cuda")
        _check("vbdr_route_records", self._L.vbdr_route_records(
            self._h, pairs.data_ptr() if n else None, n, n_ranks, recs.data_ptr(), cap,
            fill.data_ptr(), _stream_ptr(stream)))
        return recs, fill

    def apply_records(self, recs, stream=None) -> None:
        assert recs.is_cuda and recs.is_contiguous() and recs.dtype == torch_int32()
        n = recs.numel()
        _check("vbdr_apply_records", self._L.vbdr_apply_records(
            self._h, recs.data_ptr() if n else None, n, _stream_ptr(stream)))

    def registers_device(self):
        """A copy (uint8 CUDA tensor) of the registers of the last slide."""
        _, _, reg, _ = self._pointers()
        return _device_copy(reg, self.cfg.num_bdr, "|u1")

    def pcsa_device(self):
        """A copy (uint8 CUDA tensor) of the PCSA statistics (gsmall)."""
        _, _, _, pc = self._pointers()
        assert pc, "PCSA statistics exist in the gsmall layout only"
        return _device_copy(pc, self.cfg.num_bdr, "|u1")

    def set_registers(self, reg, pcsa=None, stream=None) -> None:
        """Install registers (uint8 CUDA tensor of Z values) and, for gsmall,
        PCSA statistics; recomputes the pool sums."""
        import torch
        assert reg.is_cuda and reg.is_contiguous() and reg.dtype == torch.uint8
        assert reg.numel() == self.cfg.num_bdr
        if pcsa is not None:
            assert pcsa.is_cuda and pcsa.is_contiguous() and pcsa.numel() == self.cfg.num_bdr
        _check("vbdr_set_registers", self._L.vbdr_set_registers(
            self._h, reg.data_ptr(), pcsa.data_ptr() if pcsa is not None else None,
            _stream_ptr(stream)))

    # -- checkpoint / resume -------------------------------------------------------
    def save(self, stream=None) -> bytes:
        n = ctypes.c_uint64()
        _check("vbdr_state_bytes", self._L.vbdr_state_bytes(self._h, ctypes.byref(n)))
        buf = ctypes.create_string_buffer(n.value)
        _check("vbdr_save", self._L.vbdr_save(self._h, buf, n.value, _stream_ptr(stream)))
        return buf.raw

    def load(self, blob: bytes, stream=None) -> None:
        buf = ctypes.create_string_buffer(blob, len(blob))
        _check("vbdr_load", self._L.vbdr_load(self._h, buf, len(blob), _stream_ptr(stream)))

    # -- inspection --------------------------------------------------------------
    def state(self, stream=None) -> dict:
        Z = self.cfg.num_bdr
        dr = np.empty((Z, self.R), dtype=np.uint8)
        bs = np.empty(Z, dtype=np.uint32)
        reg = np.empty(Z, dtype=np.uint8)
        _check("vbdr_copy_state", self._L.vbdr_copy_state(
            self._h, dr.ctypes.data, bs.ctypes.data, reg.ctypes.data, _stream_ptr(stream)))
        return {"dr": dr, "bs": bs, "reg": reg}

    def registers(self, stream=None) -> np.ndarray:
        reg = np.empty(self.cfg.num_bdr, dtype=np.uint8)
        _check("vbdr_copy_state", self._L.vbdr_copy_state(
            self._h, None, None, reg.ctypes.data, _stream_ptr(stream)))
        return reg

    def pool_sums(self, stream=None) -> tuple[int, int]:
        S, V = ctypes.c_uint64(), ctypes.c_uint64()
        _check("vbdr_copy_pool_sums", self._L.vbdr_copy_pool_sums(
            self._h, ctypes.byref(S), ctypes.byref(V), _stream_ptr(stream)))
        return S.value, V.value

    def pool_sums_alt(self, stream=None) -> tuple[int, int]:
        """(sum of registers, sum of PCSA statistics) of the last slide."""
        L, P = ctypes.c_uint64(), ctypes.c_uint64()
        _check("vbdr_copy_pool_sums_alt", self._L.vbdr_copy_pool_sums_alt(
            self._h, ctypes.byref(L), ctypes.byref(P), _stream_ptr(stream)))
        return L.value, P.value

    def check_flags(self) -> tuple[int, bool]:
        """(violations recorded by the bounds-checked build, whether this
        library is that build)."""
        f, c = _U32(), ctypes.c_int()
        _check("vbdr_check_flags", self._L.vbdr_check_flags(self._h, ctypes.byref(f), ctypes.byref(c)))
        return f.value, bool(c.value)

    def pcsa_statistics(self, stream=None) -> np.ndarray:
        """PCSA statistic of every physical BDR at the last slide (gsmall)."""
        out = np.empty(self.cfg.num_bdr, dtype=np.uint8)
        _check("vbdr_copy_pcsa", self._L.vbdr_copy_pcsa(self._h, out.ctypes.data,
                                                        _stream_ptr(stream)))
        return out


class Plan:
    """A host list's map from virtual to physical registers, grouped by
    register chunk, for ``Vbdr.estimate_planned`` (see include/vbdr.h).
    Valid for every handle of the same configuration on the same device."""

    def __init__(self, L, p, n_hosts: int):
        self._L, self._p, self.n_hosts = L, p, n_hosts

    def info(self) -> dict:
        n, e, b = _U64(), _U64(), _U64()
        _check("vbdr_plan_info", self._L.vbdr_plan_info(self._p, ctypes.byref(n), ctypes.byref(e),
                                                        ctypes.byref(b)))
        return {"hosts": n.value, "entries": e.value, "device_bytes": b.value}

    def status(self) -> None:
        """Raise VbdrError if a bounded wait of an earlier estimate expired."""
        _check("vbdr_plan_status", self._L.vbdr_plan_status(self._p))

    def close(self) -> None:
        if getattr(self, "_p", None):
            self._L.vbdr_plan_destroy(self._p)
            self._p = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class server_config(ctypes.Structure):
    _fields_ = [("device_budget_bytes", ctypes.c_uint64), ("max_tenants", ctypes.c_uint32),
                ("reserved", ctypes.c_uint32)]


class Server:
    """Streaming service (see include/vbdr.h): tenants admitted under a device
    memory budget, one CUDA graph replay per slice."""

    def __init__(self, budget_bytes: int, max_tenants: int = 16):
        import torch
        if not torch.cuda.is_available():
            raise RuntimeError("the service needs a CUDA GPU")
        torch.cuda.init()
        self._L = load()
        h = ctypes.c_void_p()
        c = server_config(budget_bytes, max_tenants, 0)
        _check("vbdr_server_create", self._L.vbdr_server_create(ctypes.byref(c), ctypes.byref(h)))
        self._h = h

    def close(self) -> None:
        if getattr(self, "_h", None):
            self._L.vbdr_server_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def tenant_bytes(self, cfg: Config, max_pairs: int, n_hosts: int) -> int:
        c = cfg.to_c()
        return self._L.vbdr_server_tenant_bytes(ctypes.byref(c), max_pairs, n_hosts)

    def open(self, cfg: Config, max_pairs: int, aips: np.ndarray, mlp: "Mlp | None" = None,
             timeout_ms: int = 60000) -> int:
        aips = np.ascontiguousarray(aips, dtype=np.uint32)
        c = cfg.to_c()
        t = ctypes.c_uint32()
        _check("vbdr_server_open", self._L.vbdr_server_open(
            self._h, ctypes.byref(c), max_pairs, aips.ctypes.data, aips.size,
            mlp._h if mlp is not None else None, timeout_ms, ctypes.byref(t)))
        return t.value

    def close_tenant(self, tenant: int) -> None:
        _check("vbdr_server_close", self._L.vbdr_server_close(self._h, tenant))

    def submit(self, tenant: int, pairs) -> int:
        ptr, n = _host_ptr(pairs, 2)
        tk = ctypes.c_uint64()
        _check("vbdr_server_submit", self._L.vbdr_server_submit(self._h, tenant, ptr, n,
                                                                ctypes.byref(tk)))
        return tk.value

    def wait(self, tenant: int, ticket: int, out: np.ndarray | None = None,
             timeout_ms: int = 60000) -> tuple[float, float]:
        dms, ems = ctypes.c_float(), ctypes.c_float()
        _check("vbdr_server_wait", self._L.vbdr_server_wait(
            self._h, tenant, ticket, out.ctypes.data if out is not None else None, timeout_ms,
            ctypes.byref(dms), ctypes.byref(ems)))
        return dms.value, ems.value

    def tenant_view(self, tenant: int, cfg: Config) -> "Vbdr":
        """The tenant's state handle, borrowed from the server (inspection only,
        once every submitted slice has been waited for; valid until the
        tenant is closed)."""
        h = ctypes.c_void_p()
        _check("vbdr_server_tenant_handle", self._L.vbdr_server_tenant_handle(
            self._h, tenant, ctypes.byref(h)))
        return Vbdr(cfg, _borrowed=h)

    def in_use(self) -> tuple[int, int]:
        b, t = ctypes.c_uint64(), ctypes.c_uint32()
        _check("vbdr_server_in_use", self._L.vbdr_server_in_use(self._h, ctypes.byref(b),
                                                                ctypes.byref(t)))
        return b.value, t.value


class Mlp:
    """The learned correction's network (see include/vbdr.h): BF16/FP32
    tensor-core kernels for training and inference live in the library."""

    def __init__(self, seed: int = 1):
        import torch
        if not torch.cuda.is_available():
            raise RuntimeError("the MLP kernels need a CUDA GPU")
        self._L = load()
        h = ctypes.c_void_p()
        _check("vbdr_mlp_create", self._L.vbdr_mlp_create(seed, ctypes.byref(h)))
        self._h = h
        self.n_params = self._L.vbdr_mlp_num_params()

    def close(self) -> None:
        if getattr(self, "_h", None):
            self._L.vbdr_mlp_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def get_params(self) -> tuple[np.ndarray, float]:
        p = np.empty(self.n_params, dtype=np.float32)
        nmax = ctypes.c_float()
        _check("vbdr_mlp_get_params", self._L.vbdr_mlp_get_params(self._h, p.ctypes.data,
                                                                  ctypes.byref(nmax)))
        return p, nmax.value

    def set_params(self, params: np.ndarray, nmax: float = 3.0e38) -> None:
        p = np.ascontiguousarray(params, dtype=np.float32)
        assert p.size == self.n_params
        _check("vbdr_mlp_set_params", self._L.vbdr_mlp_set_params(self._h, p.ctypes.data, nmax))

    def train(self, X, y, epochs: int, batch: int, lr: float, weight_decay: float = 0.0,
              stream=None) -> np.ndarray:
        """X: bf16 [n, 48] CUDA tensor, y: f32 [n] CUDA tensor."""
        losses = np.zeros(epochs, dtype=np.float32)
        _check("vbdr_mlp_train", self._L.vbdr_mlp_train(
            self._h, X.data_ptr(), y.data_ptr(), y.numel(), epochs, batch, lr, weight_decay, 0,
            losses.ctypes.data, _stream_ptr(stream)))
        return losses

    def gradient(self, X, y, stream=None) -> tuple[np.ndarray, float]:
        g = np.empty(self.n_params, dtype=np.float32)
        loss = ctypes.c_float()
        _check("vbdr_mlp_gradient", self._L.vbdr_mlp_gradient(
            self._h, X.data_ptr(), y.data_ptr(), y.numel(), g.ctypes.data, ctypes.byref(loss),
            _stream_ptr(stream)))
        return g, loss.value

    def forward(self, X, stream=None):
        import torch
        n = X.shape[0]
        d = torch.empty(n, dtype=torch.float32, device=X.device)
        _check("vbdr_mlp_forward", self._L.vbdr_mlp_forward(self._h, X.data_ptr(), n,
                                                            d.data_ptr(), _stream_ptr(stream)))
        return d


class CompactNet:
    """Parameters of the compact learned correction: 465 FP32 values
    (W1 [16][10], b1, W2 [16][16], b2, w3, b3) in host memory and nmax, for
    Vbdr.estimate_planned_compact (every call passes them with its launch)."""
    N_PARAMS = 465

    def __init__(self, params: np.ndarray, nmax: float):
        params = np.ascontiguousarray(params, dtype=np.float32).reshape(-1)
        if params.size != self.N_PARAMS:
            raise ValueError(f"the compact network has {self.N_PARAMS} parameters")
        self.theta = params
        self.nmax = float(nmax)

    @classmethod
    def load(cls, path: str) -> "CompactNet":
        """From a weights file of tests/train_correction_compact.py."""
        z = np.load(path)
        return cls(z["params"], float(z["nmax"]))


def live_features(X80: np.ndarray) -> np.ndarray:
    """The 48 live columns (bins 0..31, then inputs 64..79) of 80-input rows."""
    X80 = np.asarray(X80)
    return np.ascontiguousarray(np.concatenate([X80[:, :32], X80[:, 64:80]], axis=1))


def estimate_registers_noalloc(reg, num_bdr: int, log2_g: int, seed: int, aips, out,
                               stream=None) -> None:
    """vbdr_estimate_registers_noalloc on device tensors: estimates straight
    from a register array, with no device allocation inside the library."""
    import torch
    # The C entry point cannot see buffer sizes: check them here, so that a
    # short tensor is refused instead of being read or written past its end.
    dev = torch.device("cuda", torch.cuda.current_device())
    assert reg.is_cuda and reg.device == dev and reg.is_contiguous() and reg.dtype == torch.uint8
    assert reg.numel() >= num_bdr, "reg holds fewer than num_bdr registers"
    assert aips.is_cuda and aips.device == dev and aips.is_contiguous()
    assert aips.dtype in (torch.int32, torch.uint32)
    assert out.is_cuda and out.device == dev and out.is_contiguous() and out.dtype == torch.float32
    assert out.numel() >= aips.numel(), "out is shorter than aips"
    L = load()
    n = aips.numel()
    _check("vbdr_estimate_registers_noalloc", L.vbdr_estimate_registers_noalloc(
        reg.data_ptr(), num_bdr, log2_g, seed, aips.data_ptr() if n else None, n,
        out.data_ptr() if n else None, _stream_ptr(stream)))


def torch_int32():
    import torch
    return torch.int32


def torch_uint32():
    import torch
    return torch.uint32


class _DeviceView:
    """A library-owned device buffer seen through the CUDA array interface."""

    def __init__(self, ptr: int, n: int, typestr: str):
        self.__cuda_array_interface__ = {"shape": (n,), "typestr": typestr,
                                         "data": (ptr, False), "version": 3, "strides": None}


def _device_copy(ptr: int, n: int, typestr: str):
    """A torch copy of n elements of a library-owned device buffer."""
    import torch
    torch.cuda.synchronize()
    return torch.as_tensor(_DeviceView(ptr, n, typestr), device="cuda").clone()


def _host_ptr(a, width: int):
    """(pointer, element count / width) of a C-contiguous host array."""
    if isinstance(a, np.ndarray):
        assert a.flags["C_CONTIGUOUS"]
        return (a.ctypes.data if a.size else None), a.size // width
    assert not a.is_cuda and a.is_contiguous()
    return (a.data_ptr() if a.numel() else None), a.numel() // width
