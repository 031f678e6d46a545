"""Thin Python binding of libhsma (the C ABI in include/hsma.h).

Argument marshalling only: every step of the method runs in the library's
CUDA kernels.  Device arrays are torch CUDA tensors (PyTorch provides device
memory and streams); host arrays are numpy arrays.  If the library has not
been built this module raises -- there is no fallback path.
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libhsma.so")

HSMA_OK = 0
PERIODIC, GROUNDED = 0, 1
FP64, FP32_ACC64, FP32_TC_FIT = 0, 1, 2
PRECISIONS = {"fp64": FP64, "fp32": FP32_ACC64, "fp32_tc": FP32_TC_FIT}


class HsmaError(RuntimeError):
    """A negative return code of the C ABI, with its hsma_strerror text.
    ``status``: for a failed batched call, each system's own code (numpy
    int32 array), else None."""
    def __init__(self, code: int, where: str, status=None):
        self.code = code
        self.status = status
        msg = _lib().hsma_strerror(code).decode() if _LIB is not None else str(code)
        super().__init__(f"{where}: {msg} (code {code})")


class hsma_opts(ctypes.Structure):
    """Mirror of hsma_opts (include/hsma.h)."""
    _fields_ = [("precision", ctypes.c_int), ("dr_rel", ctypes.c_double), ("fib_F2", ctypes.c_int),
                ("far_field", ctypes.c_int), ("stream", ctypes.c_void_p), ("use_graphs", ctypes.c_int),
                ("profile", ctypes.c_int)]


class hsma_particles(ctypes.Structure):
    """Mirror of hsma_particles (include/hsma.h)."""
    _fields_ = [("n", ctypes.c_int64), ("xyz", ctypes.c_void_p), ("q", ctypes.c_void_p),
                ("on_device", ctypes.c_int)]


class hsma_out(ctypes.Structure):
    """Mirror of hsma_out (include/hsma.h)."""
    _fields_ = [("energy", ctypes.c_double), ("forces", ctypes.c_void_p), ("potentials", ctypes.c_void_p),
                ("n_inset", ctypes.c_int64), ("n_images", ctypes.c_int)]


class hsma_tuning(ctypes.Structure):
    """Mirror of hsma_tuning (include/hsma.h)."""
    _fields_ = [("pair_variant", ctypes.c_int), ("items_per_slot", ctypes.c_int), ("ms", ctypes.c_double)]


class hsma_plan_info_t(ctypes.Structure):
    """Mirror of hsma_plan_info_t (include/hsma.h)."""
    _fields_ = [("bc", ctypes.c_int), ("p", ctypes.c_int), ("n_basis", ctypes.c_int), ("n_cols", ctypes.c_int),
                ("Kmon", ctypes.c_int), ("n_mon_targets", ctypes.c_int), ("F2", ctypes.c_int),
                ("F1", ctypes.c_int), ("n_images", ctypes.c_int), ("n_shifts", ctypes.c_int),
                ("Rs", ctypes.c_double), ("R0", ctypes.c_double), ("alpha", ctypes.c_double),
                ("dr", ctypes.c_double), ("cond_estimate", ctypes.c_double), ("precision", ctypes.c_int)]


# Every exported entry point with its ctypes signature (the tests check this
# list against include/hsma.h).
_VP, _I, _I64, _D = ctypes.c_void_p, ctypes.c_int, ctypes.c_int64, ctypes.c_double
SIGNATURES = {
    "hsma_opts_default": (_I, [ctypes.POINTER(hsma_opts)]),
    "hsma_plan": (_I, [ctypes.POINTER(_VP), ctypes.POINTER(_D), _I, _I, _D, _I, _I, ctypes.POINTER(hsma_opts)]),
    "hsma_plan_destroy": (None, [_VP]),
    "hsma_plan_get_info": (_I, [_VP, ctypes.POINTER(hsma_plan_info_t)]),
    "hsma_plan_dims": (_I, [ctypes.POINTER(_D), _I, _I, _D, _I, _I, ctypes.POINTER(hsma_opts),
                            ctypes.POINTER(hsma_plan_info_t)]),
    "hsma_plan_set_stream": (_I, [_VP, _VP]),
    "hsma_plan_set_precision": (_I, [_VP, _I]),
    "hsma_plan_footprint": (_I, [_VP, _I64, ctypes.POINTER(ctypes.c_size_t)]),
    "hsma_plan_get_matrix": (_I, [_VP, _I, _VP, _I64]),
    "hsma_energy_forces": (_I, [_VP, ctypes.POINTER(hsma_particles), ctypes.POINTER(hsma_out)]),
    "hsma_energy_forces_batched": (_I, [_VP, _I, _VP, ctypes.POINTER(hsma_particles), _VP, _VP, _VP, _VP]),
    "hsma_coulomb_sum": (_I, [_I64, _VP, _I64, _VP, _VP, _VP, _I, _VP]),
    "hsma_coulomb_sum_static": (_I, [_I64, _VP, _I64, _VP, _VP, _VP, _I, _VP]),
    "hsma_basis": (_I, [_I, _D, _I64, _VP, _VP, _I, _VP]),
    "hsma_strerror": (ctypes.c_char_p, [_I]),
    "hsma_version": (ctypes.c_char_p, []),
    "hsma_kernel_launches": (_I64, []),
    "hsma_allocation_calls": (_I64, []),
    "hsma_plan_set_inset_skin": (_I, [_VP, _D]),
    "hsma_plan_set_preemptible": (_I, [_VP, _I]),
    "hsma_plan_inset_stats": (_I, [_VP, ctypes.POINTER(_I64), ctypes.POINTER(_I64), ctypes.POINTER(_I64)]),
    "hsma_fp32_peak": (_I, [_VP, _VP]),
    "hsma_last_timings": (_I, [_VP, _VP, _I]),
    "hsma_last_get": (_I64, [_VP, _I, _VP, _I64]),
    "hsma_plan_set_tuning": (_I, [_VP, ctypes.POINTER(hsma_tuning)]),
    "hsma_plan_get_tuning": (_I, [_VP, _I, _VP, ctypes.POINTER(hsma_tuning)]),
    "hsma_autotune": (_I, [_VP, _I, _VP, ctypes.POINTER(hsma_particles), ctypes.c_char_p,
                           ctypes.POINTER(hsma_tuning)]),
    "hsma_plan_load_tuning": (_I, [_VP, ctypes.c_char_p]),
    "hsma_shard_near": (_I, [_VP, ctypes.POINTER(hsma_particles), _I, _I, _VP, _VP, _VP,
                             ctypes.POINTER(_I64), _VP]),
    "hsma_shard_far": (_I, [_VP, ctypes.POINTER(hsma_particles), _VP, _VP, _VP, _I64, _I, _I, _VP, _VP, _VP,
                            ctypes.POINTER(_I64), ctypes.POINTER(ctypes.c_double)]),
}

_LIB = None


def _lib():
    global _LIB
    if _LIB is None:
        if not os.path.exists(LIB_PATH):
            raise RuntimeError(f"libhsma.so is not built ({LIB_PATH}); run __graft_entry__.build() or "
                               "python -m paper_1806_04801_gb300.build")
        lib = ctypes.CDLL(LIB_PATH)
        for name, (res, args) in SIGNATURES.items():
            f = getattr(lib, name)
            f.restype = res
            f.argtypes = args
        _LIB = lib
    return _LIB


def lib():
    """The loaded library (ctypes.CDLL)."""
    return _lib()


def _check(code, where):
    if code != HSMA_OK:
        raise HsmaError(code, where)


def _is_torch(a):
    return type(a).__module__.startswith("torch")


def _ptr_and_dev(a):
    """(address, on device) of a contiguous float64 torch tensor or numpy
    array; a CUDA tensor must live on the current device (the library's
    kernels run there)."""
    if _is_torch(a):
        import torch
        if not a.is_contiguous() or a.dtype != torch.float64:
            raise ValueError("tensors must be contiguous float64")
        if a.is_cuda and a.device.index != torch.cuda.current_device():
            raise ValueError(f"tensor on {a.device}, but the current CUDA device is {torch.cuda.current_device()}")
        return a.data_ptr(), bool(a.is_cuda)
    if not (isinstance(a, np.ndarray) and a.dtype == np.float64 and a.flags.c_contiguous):
        raise ValueError("arrays must be C-contiguous float64 numpy arrays")
    return a.ctypes.data, False


def _system_arrays(xyz, q, n=None):
    """Addresses of positions (n, 3) and charges (n,), both host or both
    device, with n = len(q) unless given; returns (p_xyz, p_q, on_device, n)."""
    pxyz, dev = _ptr_and_dev(xyz)
    pq, dev2 = _ptr_and_dev(q)
    if dev != dev2:
        raise ValueError("xyz and q must both be host or both device arrays")
    n = int(q.shape[0]) if n is None else int(n)
    if tuple(q.shape) != (n,) or tuple(xyz.shape) != (n, 3):
        raise ValueError(f"expected xyz of shape ({n}, 3) and q of shape ({n},); got {tuple(xyz.shape)} and "
                         f"{tuple(q.shape)}")
    return pxyz, pq, dev, n


def _offsets(offsets, n=None):
    """Batch offsets as a contiguous int64 array of nsys + 1 entries, ending
    at n when n is given (the library itself rejects a first entry other than
    0 and empty or decreasing systems, with HSMA_E_ARG)."""
    off = np.ascontiguousarray(offsets, dtype=np.int64)
    if off.ndim != 1 or off.shape[0] < 2:
        raise ValueError("offsets must hold nsys + 1 >= 2 entries")
    if n is not None and int(off[-1]) != int(n):
        raise ValueError(f"offsets end at {int(off[-1])}, but the arrays hold {int(n)} particles")
    return off


def _precision_code(precision) -> int:
    """hsma_precision code of a name ("fp64", "fp32", "fp32_tc") or a code."""
    if isinstance(precision, str):
        if precision not in PRECISIONS:
            raise ValueError(f"precision must be one of {sorted(PRECISIONS)}, not {precision!r}")
        return PRECISIONS[precision]
    return int(precision)


def _stream_handle(stream):
    if stream is None:
        return None
    if hasattr(stream, "cuda_stream"):
        return ctypes.c_void_p(stream.cuda_stream)
    return ctypes.c_void_p(int(stream))


def kernel_launches() -> int:
    """hsma_kernel_launches: kernels this library has launched (graph nodes counted on replay)."""
    return int(_lib().hsma_kernel_launches())


def allocation_calls() -> int:
    """hsma_allocation_calls: device and pinned-host allocation and free calls this library has made."""
    return int(_lib().hsma_allocation_calls())


def fp32_peak() -> tuple:
    """hsma_fp32_peak: measured (scalar, packed) FP32 lane FMAs per second of
    the current device."""
    sc, pk = ctypes.c_double(0.0), ctypes.c_double(0.0)
    rc = _lib().hsma_fp32_peak(ctypes.byref(sc), ctypes.byref(pk))
    if rc != 0:
        raise HsmaError(rc, "hsma_fp32_peak")
    return sc.value, pk.value


def plan_dims(box, bc: int, p: int, R: float, Q: int, Kmon: int, precision=FP32_ACC64, dr_rel: float = 0.0,
              fib_F2: int = 0) -> dict:
    """hsma_plan_dims: the sizes a plan with these arguments would have (the
    fields of Plan.info() but cond_estimate), on the host, without a device."""
    o = hsma_opts()
    _check(_lib().hsma_opts_default(ctypes.byref(o)), "hsma_opts_default")
    o.precision = _precision_code(precision)
    o.dr_rel = float(dr_rel)
    o.fib_F2 = int(fib_F2)
    box_arr = (ctypes.c_double * 3)(*[float(b) for b in box])
    i = hsma_plan_info_t()
    _check(_lib().hsma_plan_dims(box_arr, int(bc), int(p), float(R), int(Q), int(Kmon), ctypes.byref(o),
                                 ctypes.byref(i)), "hsma_plan_dims")
    return {k: getattr(i, k) for k, _ in hsma_plan_info_t._fields_}


def version() -> str:
    """hsma_version."""
    return _lib().hsma_version().decode()


def strerror(code: int) -> str:
    """hsma_strerror: the message of a return code."""
    return _lib().hsma_strerror(int(code)).decode()


class Plan:
    """hsma_plan: preparation step; device-resident matrices."""

    def __init__(self, box, bc: int, p: int, R: float, Q: int, Kmon: int, precision=FP32_ACC64,
                 dr_rel: float = 0.0, fib_F2: int = 0, stream=None, profile: bool = False, use_graphs: bool = True,
                 far_field: str = "images"):
        L = _lib()
        o = hsma_opts()
        _check(L.hsma_opts_default(ctypes.byref(o)), "hsma_opts_default")
        o.precision = _precision_code(precision)
        o.dr_rel = float(dr_rel)
        o.fib_F2 = int(fib_F2)
        o.stream = _stream_handle(stream)
        o.profile = 1 if profile else 0
        o.use_graphs = 1 if use_graphs else 0
        o.far_field = {"images": 0, "series": 1}[far_field]
        box_arr = (ctypes.c_double * 3)(*[float(b) for b in box])
        h = ctypes.c_void_p()
        _check(L.hsma_plan(ctypes.byref(h), box_arr, int(bc), int(p), float(R), int(Q), int(Kmon), ctypes.byref(o)),
               "hsma_plan")
        self._h = h
        self.box = tuple(float(b) for b in box)
        codes = {v: k for k, v in PRECISIONS.items()}
        self.precision = codes.get(o.precision, str(o.precision))  # "fp64", "fp32" or "fp32_tc"

    # ------------------------------------------------------------- info
    @property
    def handle(self):
        """The opaque hsma_plan_t."""
        return self._h

    def info(self) -> dict:
        """hsma_plan_get_info: sizes the plan chose (F2, N_o, monitoring targets, shifts, ...)."""
        i = hsma_plan_info_t()
        _check(_lib().hsma_plan_get_info(self._h, ctypes.byref(i)), "hsma_plan_get_info")
        return {k: getattr(i, k) for k, _ in hsma_plan_info_t._fields_}

    def set_stream(self, stream):
        """hsma_plan_set_stream: the CUDA stream of later calls (torch stream or handle)."""
        _check(_lib().hsma_plan_set_stream(self._h, _stream_handle(stream)), "hsma_plan_set_stream")

    def set_precision(self, precision):
        """hsma_plan_set_precision: "fp64", "fp32" or "fp32_tc" for later calls."""
        _check(_lib().hsma_plan_set_precision(self._h, _precision_code(precision)), "hsma_plan_set_precision")

    def footprint(self, n: int) -> int:
        """hsma_plan_footprint: device bytes one call with n particles needs."""
        b = ctypes.c_size_t()
        _check(_lib().hsma_plan_footprint(self._h, int(n), ctypes.byref(b)), "hsma_plan_footprint")
        return int(b.value)

    def get_matrix(self, which: int) -> np.ndarray:
        """hsma_plan_get_matrix: a plan matrix copied to the host (see the header)."""
        info = self.info()
        shapes = {0: (info["n_mon_targets"], 3), 1: (info["Kmon"], info["n_cols"]),
                  2: (info["n_cols"], info["Kmon"]), 3: (2 * (info["F2"] + 1), 3), 4: (2 * (info["F2"] + 1),),
                  5: (2 * (info["F2"] + 1), info["n_basis"])}
        out = np.empty(shapes[which])
        _check(_lib().hsma_plan_get_matrix(self._h, int(which), out.ctypes.data, out.size), "hsma_plan_get_matrix")
        return out

    def last_get(self, which: int, count: int) -> np.ndarray:
        """hsma_last_get: an intermediate of the last update (A, b, Phi_in, Phi_out)."""
        out = np.empty(count)
        n = _lib().hsma_last_get(self._h, int(which), out.ctypes.data, count)
        if n < 0:
            raise HsmaError(int(n), "hsma_last_get")
        return out[:n]

    def last_timings(self) -> list:
        """hsma_last_timings: per-phase device milliseconds of the last update (profile plans)."""
        ms = np.zeros(8)
        n = _lib().hsma_last_timings(self._h, ms.ctypes.data, 8)
        if n < 0:
            raise HsmaError(int(n), "hsma_last_timings")
        return list(ms[:n])

    # ------------------------------------------------------------- update
    def energy_forces(self, xyz, q, forces=True, potentials=False):
        """hsma_energy_forces.  xyz (n, 3) and q (n,) float64, both numpy
        (host) or both torch CUDA tensors (device).  Returns
        (energy, forces or None, potentials or None, n_inset)."""
        pxyz, pq, dev, n = _system_arrays(xyz, q)
        f = p = None
        if dev:
            import torch
            if forces:
                f = torch.empty((n, 3), dtype=torch.float64, device=xyz.device)
            if potentials:
                p = torch.empty((n,), dtype=torch.float64, device=xyz.device)
        else:
            if forces:
                f = np.empty((n, 3))
            if potentials:
                p = np.empty(n)
        part = hsma_particles(n, pxyz, pq, 1 if dev else 0)
        out = hsma_out(0.0, _ptr_and_dev(f)[0] if f is not None else None,
                       _ptr_and_dev(p)[0] if p is not None else None, 0, 0)
        _check(_lib().hsma_energy_forces(self._h, ctypes.byref(part), ctypes.byref(out)), "hsma_energy_forces")
        return out.energy, f, p, out.n_inset

    def energy_forces_batched(self, xyz, q, offsets, forces=True, potentials=False):
        """hsma_energy_forces_batched over concatenated systems; offsets is a
        sequence of nsys+1 increasing integers.  Returns (energies, forces,
        potentials, status).  On an error the raised HsmaError carries the
        per-system codes in its ``status``."""
        off = _offsets(offsets)
        nsys = off.shape[0] - 1
        pxyz, pq, dev, n = _system_arrays(xyz, q, int(off[-1]))
        f = p = None
        if dev:
            import torch
            if forces:
                f = torch.empty((n, 3), dtype=torch.float64, device=xyz.device)
            if potentials:
                p = torch.empty((n,), dtype=torch.float64, device=xyz.device)
        else:
            if forces:
                f = np.empty((n, 3))
            if potentials:
                p = np.empty(n)
        e = np.empty(nsys)
        st = np.zeros(nsys, dtype=np.int32)
        part = hsma_particles(n, pxyz, pq, 1 if dev else 0)
        rc = _lib().hsma_energy_forces_batched(self._h, nsys, off.ctypes.data, ctypes.byref(part), e.ctypes.data,
                                               _ptr_and_dev(f)[0] if f is not None else None,
                                               _ptr_and_dev(p)[0] if p is not None else None, st.ctypes.data)
        if rc != HSMA_OK:
            raise HsmaError(rc, "hsma_energy_forces_batched", status=st)
        return e, f, p, st

    # ------------------------------------------------------ in-set reuse
    def set_inset_skin(self, skin: float):
        """hsma_plan_set_inset_skin: reuse the in-set between single-system
        steps while every particle stays within ``skin`` of the positions of
        the last build (0 switches reuse off)."""
        _check(_lib().hsma_plan_set_inset_skin(self._h, float(skin)), "hsma_plan_set_inset_skin")

    def set_preemptible(self, on: bool):
        """hsma_plan_set_preemptible: pair work as one CTA per work item."""
        _check(_lib().hsma_plan_set_preemptible(self._h, 1 if on else 0), "hsma_plan_set_preemptible")

    def inset_stats(self) -> dict:
        """hsma_plan_inset_stats: in-set lists built, steps that reused one,
        steps redone because the list was stale."""
        b, r, st = _I64(), _I64(), _I64()
        _check(_lib().hsma_plan_inset_stats(self._h, ctypes.byref(b), ctypes.byref(r), ctypes.byref(st)),
               "hsma_plan_inset_stats")
        return {"builds": b.value, "reuses": r.value, "stale": st.value}

    # ---------------------------------------------------- target sharding
    def _shard_args(self, xyz, q):
        pxyz, pq, dev, n = _system_arrays(xyz, q)
        return hsma_particles(n, pxyz, pq, 1 if dev else 0), n

    def shard_near(self, xyz, q, part: int, nparts: int):
        """hsma_shard_near: (index, phi_in, E_in, phi_mon) for this part
        (host arrays; phi_mon is zero outside the part's monitoring slice)."""
        part_s, n = self._shard_args(xyz, q)
        idx = np.empty(n, dtype=np.int64)
        phi = np.empty(n)
        fld = np.empty((n, 3))
        mon = np.empty(self.info()["n_mon_targets"])
        cnt = ctypes.c_int64()
        _check(_lib().hsma_shard_near(self._h, ctypes.byref(part_s), int(part), int(nparts), idx.ctypes.data,
                                      phi.ctypes.data, fld.ctypes.data, ctypes.byref(cnt), mon.ctypes.data),
               "hsma_shard_near")
        k = cnt.value
        return idx[:k].copy(), phi[:k].copy(), fld[:k].copy(), mon

    def shard_far(self, xyz, q, phi_mon, phi_in, e_in, part: int, nparts: int):
        """hsma_shard_far: (index, potentials, forces, energy of the part) for
        this part, from the summed monitoring potentials and the part's
        near-stage Phi_in, E_in (owned order)."""
        part_s, n = self._shard_args(xyz, q)
        mon = np.ascontiguousarray(phi_mon, dtype=np.float64)
        if mon.shape != (self.info()["n_mon_targets"],):
            raise ValueError("phi_mon must hold one value per monitoring target")
        pin = np.ascontiguousarray(phi_in, dtype=np.float64)
        ein = np.ascontiguousarray(e_in, dtype=np.float64)
        if pin.ndim != 1 or pin.shape[0] > n or ein.shape != (pin.shape[0], 3):
            raise ValueError("phi_in / e_in must be the near stage's arrays of this part (k and k x 3)")
        idx = np.empty(n, dtype=np.int64)
        pot = np.empty(n)
        frc = np.empty((n, 3))
        cnt = ctypes.c_int64()
        u = ctypes.c_double()
        _check(_lib().hsma_shard_far(self._h, ctypes.byref(part_s), mon.ctypes.data, pin.ctypes.data,
                                     ein.ctypes.data, int(pin.shape[0]), int(part), int(nparts), idx.ctypes.data,
                                     pot.ctypes.data, frc.ctypes.data, ctypes.byref(cnt), ctypes.byref(u)),
               "hsma_shard_far")
        k = cnt.value
        return idx[:k].copy(), pot[:k].copy(), frc[:k].copy(), u.value

    # ------------------------------------------------------------ tuning
    def set_tuning(self, pair_variant=None, items_per_slot=None):
        """Fix the pair kernel's work decomposition (None, None: automatic)."""
        if pair_variant is None and items_per_slot is None:
            _check(_lib().hsma_plan_set_tuning(self._h, None), "hsma_plan_set_tuning")
            return
        t = hsma_tuning(int(pair_variant or 4), int(items_per_slot or 24), 0.0)
        _check(_lib().hsma_plan_set_tuning(self._h, ctypes.byref(t)), "hsma_plan_set_tuning")

    def get_tuning(self, offsets) -> dict:
        """hsma_plan_get_tuning: the tuning a call with these offsets would use."""
        off = _offsets(offsets)
        t = hsma_tuning()
        _check(_lib().hsma_plan_get_tuning(self._h, off.shape[0] - 1, off.ctypes.data, ctypes.byref(t)),
               "hsma_plan_get_tuning")
        return {"pair_variant": t.pair_variant, "items_per_slot": t.items_per_slot, "ms": t.ms}

    def autotune(self, xyz, q, offsets=None, cache_path=None) -> dict:
        """hsma_autotune on a batch (offsets None: one system)."""
        pxyz, pq, dev, n = _system_arrays(xyz, q)
        off = _offsets([0, n] if offsets is None else offsets, n)
        part = hsma_particles(n, pxyz, pq, 1 if dev else 0)
        t = hsma_tuning()
        _check(_lib().hsma_autotune(self._h, off.shape[0] - 1, off.ctypes.data, ctypes.byref(part),
                                    cache_path.encode() if cache_path else None, ctypes.byref(t)), "hsma_autotune")
        return {"pair_variant": t.pair_variant, "items_per_slot": t.items_per_slot, "ms": t.ms}

    def load_tuning(self, cache_path) -> int:
        """hsma_plan_load_tuning: entries of an autotuner cache matching this plan; returns how many."""
        r = _lib().hsma_plan_load_tuning(self._h, str(cache_path).encode())
        if r < 0:
            raise HsmaError(r, "hsma_plan_load_tuning")
        return int(r)

    def close(self):
        """hsma_plan_destroy (idempotent)."""
        if getattr(self, "_h", None):
            _lib().hsma_plan_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()


def coulomb_sum(src, tgt, field=True, precision=FP32_ACC64, stream=None):
    """hsma_coulomb_sum on torch CUDA tensors: src (ns, 4) = (x, y, z, q),
    tgt (nt, 3).  Returns (pot, field or None)."""
    import torch
    ps, dev = _ptr_and_dev(src)
    pt, dev2 = _ptr_and_dev(tgt)
    if not (dev and dev2):
        raise ValueError("coulomb_sum takes CUDA tensors")
    if src.dim() != 2 or src.shape[1] != 4 or tgt.dim() != 2 or tgt.shape[1] != 3:
        raise ValueError("src must have shape (ns, 4) and tgt shape (nt, 3)")
    nt = tgt.shape[0]
    pot = torch.empty(nt, dtype=torch.float64, device=tgt.device)
    fld = torch.empty((nt, 3), dtype=torch.float64, device=tgt.device) if field else None
    precision = _precision_code(precision)
    _check(_lib().hsma_coulomb_sum(src.shape[0], ps, nt, pt, pot.data_ptr(),
                                   fld.data_ptr() if fld is not None else None, int(precision),
                                   _stream_handle(stream)), "hsma_coulomb_sum")
    return pot, fld


def coulomb_sum_static(src, tgt, field=True, precision=FP32_ACC64, stream=None):
    """hsma_coulomb_sum_static: the same sums with no device allocation (its
    working memory is a fixed static device array inside the library; calls
    must not overlap on the GPU).  CUDA tensors as for coulomb_sum."""
    import torch
    ps, dev = _ptr_and_dev(src)
    pt, dev2 = _ptr_and_dev(tgt)
    if not (dev and dev2):
        raise ValueError("coulomb_sum_static takes CUDA tensors")
    if src.dim() != 2 or src.shape[1] != 4 or tgt.dim() != 2 or tgt.shape[1] != 3:
        raise ValueError("src must have shape (ns, 4) and tgt shape (nt, 3)")
    nt = tgt.shape[0]
    pot = torch.empty(nt, dtype=torch.float64, device=tgt.device)
    fld = torch.empty((nt, 3), dtype=torch.float64, device=tgt.device) if field else None
    precision = _precision_code(precision)
    _check(_lib().hsma_coulomb_sum_static(src.shape[0], ps, nt, pt, pot.data_ptr(),
                                          fld.data_ptr() if fld is not None else None, int(precision),
                                          _stream_handle(stream)), "hsma_coulomb_sum_static")
    return pot, fld


def basis(pts, p: int, Rs: float, precision: str = "fp64", stream=None):
    """hsma_basis on a torch CUDA tensor of points (np, 3).  precision "fp64"
    (FP64 recurrence) or "fp32" (double-float recurrence on the FP32 pipe,
    ~1e-14 relative); the result is FP64 either way."""
    import torch
    pp, dev = _ptr_and_dev(pts)
    if not dev:
        raise ValueError("basis takes a CUDA tensor")
    if pts.dim() != 2 or pts.shape[1] != 3:
        raise ValueError("pts must have shape (np, 3)")
    out = torch.empty((pts.shape[0], (p + 1) ** 2), dtype=torch.float64, device=pts.device)
    prec = {"fp64": FP64, "fp32": FP32_ACC64}.get(precision)
    if prec is None:
        raise ValueError("basis precision is 'fp64' or 'fp32'")
    _check(_lib().hsma_basis(int(p), float(Rs), pts.shape[0], pp, out.data_ptr(), prec, _stream_handle(stream)),
           "hsma_basis")
    return out


# ------------------------------------------------------------------ serving
class hsma_server_opts(ctypes.Structure):
    """Mirror of hsma_server_opts (include/hsma.h)."""
    _fields_ = [("hbm_budget_bytes", ctypes.c_size_t), ("max_batch", ctypes.c_int), ("lanes", ctypes.c_int),
                ("precision", ctypes.c_int), ("express_lanes", ctypes.c_int), ("express_max_n", ctypes.c_int64),
                ("mid_lanes", ctypes.c_int), ("mid_max_n", ctypes.c_int64)]


class hsma_request_info(ctypes.Structure):
    """Mirror of hsma_request_info (include/hsma.h)."""
    _fields_ = [("n", ctypes.c_int64), ("latency_ms", ctypes.c_double), ("queue_ms", ctypes.c_double),
                ("batch_size", ctypes.c_int), ("status", ctypes.c_int)]


class hsma_server_stats_t(ctypes.Structure):
    """Mirror of hsma_server_stats_t (include/hsma.h)."""
    _fields_ = [("completed", ctypes.c_int64), ("failed", ctypes.c_int64), ("cancelled", ctypes.c_int64),
                ("queued", ctypes.c_int64),
                ("batches", ctypes.c_int64), ("mean_batch", ctypes.c_double), ("elapsed_s", ctypes.c_double),
                ("hbm_held_bytes", ctypes.c_size_t), ("hbm_budget_bytes", ctypes.c_size_t)]


SIGNATURES.update({
    "hsma_server_opts_default": (_I, [ctypes.POINTER(hsma_server_opts)]),
    "hsma_server_create": (_I, [ctypes.POINTER(_VP), ctypes.POINTER(_D), _I, _I, _D, _I, _I,
                                ctypes.POINTER(hsma_server_opts)]),
    "hsma_server_submit": (_I, [_VP, _I64, _VP, _VP, ctypes.POINTER(_I64)]),
    "hsma_server_result": (_I, [_VP, _I64, _I, ctypes.POINTER(_D), _VP, ctypes.POINTER(hsma_request_info)]),
    "hsma_server_stats": (_I, [_VP, ctypes.POINTER(hsma_server_stats_t)]),
    "hsma_server_cancel": (_I, [_VP, _I64]),
    "hsma_server_destroy": (None, [_VP]),
})


class Server:
    """hsma_server_*: continuous-batching request loop over resident plans."""

    def __init__(self, box, bc: int, p: int, R: float, Q: int, Kmon: int, precision=FP32_ACC64, lanes: int = 2,
                 max_batch: int = 64, hbm_budget_bytes: int = 0, express_lanes: int | None = None,
                 express_max_n: int | None = None, mid_lanes: int = 0, mid_max_n: int | None = None):
        L = _lib()
        o = hsma_server_opts()
        _check(L.hsma_server_opts_default(ctypes.byref(o)), "hsma_server_opts_default")
        o.precision = _precision_code(precision)
        o.lanes = int(lanes)
        o.max_batch = int(max_batch)
        o.hbm_budget_bytes = int(hbm_budget_bytes)
        if express_lanes is not None:
            o.express_lanes = int(express_lanes)
        else:  # the default, as far as lanes allow (one lane at least is bulk)
            o.express_lanes = min(int(o.express_lanes), int(lanes) - 1)
        if express_max_n is not None:
            o.express_max_n = int(express_max_n)
        o.mid_lanes = int(mid_lanes)
        if mid_max_n is not None:
            o.mid_max_n = int(mid_max_n)
        box_arr = (ctypes.c_double * 3)(*[float(b) for b in box])
        h = ctypes.c_void_p()
        _check(L.hsma_server_create(ctypes.byref(h), box_arr, int(bc), int(p), float(R), int(Q), int(Kmon),
                                    ctypes.byref(o)), "hsma_server_create")
        self._h = h
        self._sizes = {}  # ticket -> particles, so result() sizes the force buffer itself

    def submit(self, xyz: np.ndarray, q: np.ndarray) -> int:
        """hsma_server_submit: queue one configuration (host arrays); returns its ticket."""
        xyz = np.ascontiguousarray(xyz, dtype=np.float64)
        q = np.ascontiguousarray(q, dtype=np.float64)
        if q.ndim != 1 or xyz.shape != (q.shape[0], 3):
            raise ValueError(f"expected xyz of shape ({q.shape[0]}, 3) and q of shape (n,)")
        t = ctypes.c_int64()
        _check(_lib().hsma_server_submit(self._h, q.shape[0], xyz.ctypes.data, q.ctypes.data, ctypes.byref(t)),
               "hsma_server_submit")
        self._sizes[int(t.value)] = int(q.shape[0])
        return int(t.value)

    def result(self, ticket: int, n: int | None = None, wait: bool = True, forces: bool = True):
        """(code, energy, forces or None, info dict); code HSMA_E_AGAIN (-10)
        when not ready and wait is False.  The force buffer is sized from the
        submitted request (n, if given, must agree with it)."""
        ticket = int(ticket)
        n_sub = self._sizes.get(ticket)
        if n is not None and n_sub is not None and int(n) != n_sub:
            raise ValueError(f"ticket {ticket} holds {n_sub} particles, not {n}")
        n = n_sub if n_sub is not None else n
        e = ctypes.c_double()
        info = hsma_request_info()
        f = np.empty((n, 3)) if (forces and n) else None
        code = _lib().hsma_server_result(self._h, ticket, 1 if wait else 0, ctypes.byref(e),
                                         f.ctypes.data if f is not None else None, ctypes.byref(info))
        if code != -10:  # collected (or unknown): the ticket is gone
            self._sizes.pop(ticket, None)
        return code, e.value, f, {k: getattr(info, k) for k, _ in hsma_request_info._fields_}

    def cancel(self, ticket: int) -> int:
        """hsma_server_cancel: 0 if withdrawn, -10 if already running/ran."""
        return int(_lib().hsma_server_cancel(self._h, int(ticket)))

    def stats(self) -> dict:
        """hsma_server_stats: counts of queued, running, completed, failed and cancelled requests."""
        st = hsma_server_stats_t()
        _check(_lib().hsma_server_stats(self._h, ctypes.byref(st)), "hsma_server_stats")
        return {k: getattr(st, k) for k, _ in hsma_server_stats_t._fields_}

    def close(self):
        if getattr(self, "_h", None):
            _lib().hsma_server_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()
