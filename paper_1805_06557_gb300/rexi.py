"""ctypes binding of librexi.so (argument marshalling only; every step runs in the library).

Importing this module loads the library and raises ImportError if it has not been built
(``python -c "import __graft_entry__ as g; g.build()"``).  There is no fallback path.
"""
import ctypes
import os
import re

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "librexi.so")
HEADER_DIR = os.path.join(os.path.dirname(_HERE), "include")

if not os.path.exists(LIB_PATH):
    raise ImportError("librexi.so is not built (%s); run __graft_entry__.build()" % LIB_PATH)
_lib = ctypes.CDLL(LIB_PATH)

REXI_OK, REXI_EINVAL, REXI_ENOMEM, REXI_ECUDA, REXI_ETIMEOUT, REXI_EBUSY = 0, -1, -2, -3, -4, -5
REXI_FP64, REXI_MIXED = 0, 1
_PREC = {"fp64": REXI_FP64, "mixed": REXI_MIXED}
REXI_PART_NONE, REXI_PART_POLES, REXI_PART_M = 0, 1, 2
_PART = {None: REXI_PART_NONE, "none": REXI_PART_NONE, "poles": REXI_PART_POLES, "m": REXI_PART_M}


class RexiError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__("%s (code %d)" % (msg, code))
        self.code = code


def _check(rc):
    if rc != REXI_OK:
        raise RexiError(rc, _lib.rexi_last_error().decode())
    return rc


_dp = ctypes.POINTER(ctypes.c_double)
_ip = ctypes.POINTER(ctypes.c_int)


class PlanDesc(ctypes.Structure):
    _fields_ = [("T", ctypes.c_int), ("N", ctypes.c_int), ("dt", ctypes.c_double),
                ("omega", ctypes.c_double), ("radius", ctypes.c_double),
                ("phibar", ctypes.c_double), ("p0", ctypes.c_double), ("Xc", ctypes.c_double),
                ("z", _dp), ("w", _dp), ("precision", ctypes.c_int),
                ("heavy_tau", ctypes.c_double), ("max_batch", ctypes.c_int),
                ("stream", ctypes.c_void_p), ("prune_tau", ctypes.c_double),
                ("part_mode", ctypes.c_int), ("part_rank", ctypes.c_int), ("part_size", ctypes.c_int),
                ("fp64_tau", ctypes.c_double)]


class PlanInfo(ctypes.Structure):
    _fields_ = [("T", ctypes.c_int), ("N", ctypes.c_int), ("nlm", ctypes.c_int),
                ("precision", ctypes.c_int), ("n_heavy", ctypes.c_int),
                ("n_groups", ctypes.c_int), ("n_tiles", ctypes.c_int), ("q_slots", ctypes.c_int),
                ("grid_fp64", ctypes.c_int), ("grid_light", ctypes.c_int),
                ("grid_heavy", ctypes.c_int), ("workspace_bytes", ctypes.c_longlong),
                ("s0_re", ctypes.c_double), ("s0_im", ctypes.c_double), ("X", ctypes.c_double),
                ("n_pruned", ctypes.c_int), ("pruned_gain", ctypes.c_double), ("n_fp64", ctypes.c_int)]


_lib.rexi_last_error.restype = ctypes.c_char_p
_lib.rexi_coeffs.argtypes = [ctypes.c_int, ctypes.c_double, ctypes.c_double, ctypes.c_int, _dp, _dp]
_lib.rexi_contour_select.argtypes = [ctypes.c_double, ctypes.c_int, _dp, _dp]
_lib.rexi_select_poles.argtypes = [ctypes.c_int, ctypes.c_int, _dp, _dp, ctypes.c_double, ctypes.c_double,
                                   ctypes.c_double, ctypes.c_int, _ip, _dp]
_lib.rexi_spectrum_bound.argtypes = [ctypes.c_int] + [ctypes.c_double] * 4
_lib.rexi_spectrum_bound.restype = ctypes.c_double
_lib.rexi_plan_create.argtypes = [ctypes.POINTER(PlanDesc), ctypes.POINTER(ctypes.c_void_p)]
_lib.rexi_plan_destroy.argtypes = [ctypes.c_void_p]
_lib.rexi_step.argtypes = [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int]
_lib.rexi_step_host.argtypes = [ctypes.c_void_p, _dp, _dp, ctypes.c_int]
_lib.rexi_step_host_async.argtypes = [ctypes.c_void_p, _dp, _dp, ctypes.c_int]
_lib.rexi_sync.argtypes = [ctypes.c_void_p]
_lib.rexi_plan_get_info.argtypes = [ctypes.c_void_p, ctypes.POINTER(PlanInfo)]
_lib.rexi_plan_get_poles.argtypes = [ctypes.c_void_p, _dp, _dp, _ip]
_lib.rexi_alu_peaks.argtypes = [_dp, _dp]
_lib.rexi_partition.argtypes = [ctypes.c_int] * 5 + [_ip]


def partition(mode, T, N, rank, size):
    """Which poles (mode "poles": N entries) or zonal orders (mode "m": T + 1 entries) rank
    `rank` of `size` owns, as a boolean array (include/rexi.h rexi_partition)."""
    n = int(N) if mode == "poles" else int(T) + 1
    own = np.zeros(n, dtype=np.int32)
    _check(_lib.rexi_partition(_PART[mode], int(T), int(N), int(rank), int(size), own.ctypes.data_as(_ip)))
    return own.astype(bool)


def step_allreduce(plan, U0, U1, group=None):
    """One step of a partitioned plan on every rank, completed by a sum all-reduce of U1 over the
    ranks of `group` (torch.distributed; NCCL on GPUs): each rank's U1 holds its share (a partial
    pole sum, or its zonal orders and zeros), and the sum is the whole step."""
    import torch
    import torch.distributed as dist
    plan.step(U0, U1)
    dist.all_reduce(torch.view_as_real(U1), op=dist.ReduceOp.SUM, group=group)
    return U1
_lib.rexi_plan_set_profiling.argtypes = [ctypes.c_void_p, ctypes.c_int]
_lib.rexi_plan_get_profile.argtypes = [ctypes.c_void_p, _dp, _ip, ctypes.c_int]
_lib.rexi_step_fp64_static.argtypes = [ctypes.c_int, ctypes.c_int] + [ctypes.c_double] * 6 + \
    [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p]
_lib.rexi_static_scratch_bytes.restype = ctypes.c_longlong


def _dev_tensor(t, numel, dtype, what, at_least=False):
    """Checks that `t` is a contiguous CUDA tensor of `dtype` on the current device holding
    `numel` elements (at least `numel` with at_least) before its address reaches a kernel:
    a wrong size, stride or device would make the kernel read or write outside the buffer."""
    import torch
    dt = getattr(torch, dtype)
    if not isinstance(t, torch.Tensor):
        raise ValueError("%s: need a torch tensor, got %s" % (what, type(t).__name__))
    if t.dtype != dt:
        raise ValueError("%s: need dtype %s, got %s" % (what, dtype, t.dtype))
    if not t.is_contiguous():
        raise ValueError("%s: need a contiguous tensor" % what)
    if (t.numel() < numel) if at_least else (t.numel() != numel):
        raise ValueError("%s: need %s%d elements, got %d" % (what, "at least " if at_least else "",
                                                           numel, t.numel()))
    if not t.is_cuda:
        raise ValueError("%s: need a CUDA tensor, got one on %s" % (what, t.device))
    if t.device.index != torch.cuda.current_device():
        raise ValueError("%s: tensor on %s, current device is cuda:%d"
                         % (what, t.device, torch.cuda.current_device()))
    return ctypes.c_void_p(t.data_ptr())


def step_fp64_static(T, N, dt, omega, radius, phibar, p0, Xc, U0, U1, stream=None):
    """Allocation-free FP64 REXI step on one state (CUDA complex128 tensors [3, nlm])."""
    n = 3 * nlm(int(T)) if int(T) >= 0 else 0
    p0_ = _dev_tensor(U0, n, "complex128", "U0")
    p1_ = _dev_tensor(U1, n, "complex128", "U1")
    _check(_lib.rexi_step_fp64_static(int(T), int(N), float(dt), float(omega), float(radius),
                                      float(phibar), float(p0), float(Xc), p0_, p1_,
                                      ctypes.c_void_p(_stream_handle(stream))))
    return U1


def static_scratch_bytes():
    return int(_lib.rexi_static_scratch_bytes())


class RaggedDesc(ctypes.Structure):
    _fields_ = [("Tmax", ctypes.c_int), ("max_inst", ctypes.c_int), ("max_poles", ctypes.c_int),
                ("max_elems", ctypes.c_longlong), ("omega", ctypes.c_double),
                ("radius", ctypes.c_double), ("phibar", ctypes.c_double),
                ("precision", ctypes.c_int), ("heavy_tau", ctypes.c_double),
                ("stream", ctypes.c_void_p), ("prune_tau", ctypes.c_double), ("fp64_tau", ctypes.c_double)]


class Instance(ctypes.Structure):
    _fields_ = [("T", ctypes.c_int), ("N", ctypes.c_int), ("dt", ctypes.c_double),
                ("p0", ctypes.c_double), ("Xc", ctypes.c_double), ("soff", ctypes.c_longlong)]


_lib.rexi_ragged_create.argtypes = [ctypes.POINTER(RaggedDesc), ctypes.POINTER(ctypes.c_void_p)]
_lib.rexi_ragged_destroy.argtypes = [ctypes.c_void_p]
_lib.rexi_ragged_set.argtypes = [ctypes.c_void_p, ctypes.c_int, ctypes.POINTER(Instance)]
_lib.rexi_ragged_offsets.argtypes = [ctypes.c_void_p, ctypes.POINTER(ctypes.c_longlong)]
_lib.rexi_ragged_step.argtypes = [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p]
_lib.rexi_ragged_capture.argtypes = [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p]
_lib.rexi_ragged_tune.argtypes = [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int,
                                  _ip, _dp]
_lib.rexi_ragged_sync.argtypes = [ctypes.c_void_p]
_lib.rexi_ragged_set_profiling.argtypes = [ctypes.c_void_p, ctypes.c_int]
_lib.rexi_ragged_get_profile.argtypes = [ctypes.c_void_p, _dp, _ip, ctypes.c_int]


class RaggedPlan:
    """One REXI launch over states of different truncation, time step and pole count."""

    def __init__(self, Tmax, max_inst, max_poles, max_elems, omega, radius, phibar,
                 precision="mixed", heavy_tau=-1.0, prune_tau=0.0, stream=None, fp64_tau=0.0):
        d = RaggedDesc()
        d.Tmax, d.max_inst, d.max_poles, d.max_elems = int(Tmax), int(max_inst), int(max_poles), int(max_elems)
        d.omega, d.radius, d.phibar = float(omega), float(radius), float(phibar)
        d.precision = _PREC[precision] if isinstance(precision, str) else int(precision)
        d.heavy_tau = float(heavy_tau)
        d.prune_tau = float(prune_tau)
        d.fp64_tau = float(fp64_tau)
        d.stream = ctypes.c_void_p(_stream_handle(stream))
        h = ctypes.c_void_p()
        _check(_lib.rexi_ragged_create(ctypes.byref(d), ctypes.byref(h)))
        self._h = h
        self.n = 0

    def set(self, instances):
        """instances: iterable of (T, N, dt, p0, Xc) or (T, N, dt, p0, Xc, soff); returns the
        complex offsets of the states (and the extent as the last entry)."""
        arr = (Instance * len(instances))()
        for i, inst in enumerate(instances):
            T, N, dt, p0, Xc = inst[:5]
            arr[i].T, arr[i].N, arr[i].dt, arr[i].p0, arr[i].Xc = int(T), int(N), float(dt), float(p0), float(Xc)
            arr[i].soff = int(inst[5]) if len(inst) > 5 else -1
        _check(_lib.rexi_ragged_set(self._h, len(instances), arr))
        self.n = len(instances)
        return self.offsets()

    def offsets(self):
        o = (ctypes.c_longlong * (self.n + 1))()
        _check(_lib.rexi_ragged_offsets(self._h, o))
        return [int(v) for v in o]

    def _states(self, U0, U1):
        n = self.offsets()[-1]
        return (_dev_tensor(U0, n, "complex128", "U0", at_least=True),
                _dev_tensor(U1, n, "complex128", "U1", at_least=True))

    def step(self, U0, U1):
        _check(_lib.rexi_ragged_step(self._h, *self._states(U0, U1)))
        return U1

    def capture(self, U0, U1):
        _check(_lib.rexi_ragged_capture(self._h, *self._states(U0, U1)))

    def tune(self, U0, U1, reps=3):
        q = ctypes.c_int()
        ms = ctypes.c_double()
        _check(_lib.rexi_ragged_tune(self._h, *self._states(U0, U1), int(reps), ctypes.byref(q),
                                     ctypes.byref(ms)))
        return q.value, ms.value

    def sync(self):
        _check(_lib.rexi_ragged_sync(self._h))

    def set_profiling(self, enable=True):
        _check(_lib.rexi_ragged_set_profiling(self._h, 1 if enable else 0))

    def profile(self, reset=True):
        ms = np.zeros(len(KERNEL_NAMES))
        n = np.zeros(len(KERNEL_NAMES), dtype=np.int32)
        _check(_lib.rexi_ragged_get_profile(self._h, ms.ctypes.data_as(_dp), n.ctypes.data_as(_ip),
                                            1 if reset else 0))
        return {k: (float(ms[i]), int(n[i])) for i, k in enumerate(KERNEL_NAMES)}

    def close(self):
        if getattr(self, "_h", None) is not None and self._h.value:
            _lib.rexi_ragged_destroy(self._h)
            self._h = ctypes.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


KERNEL_NAMES = ["k_mixed_rhs", "k_rexi_fp64", "k_rexi_light", "k_rexi_heavy", "k_rexi_finalize"]


def alu_peaks():
    """Measured (FP64, FP32) FMA throughput of the current device in TFLOP/s."""
    a = ctypes.c_double()
    b = ctypes.c_double()
    _check(_lib.rexi_alu_peaks(ctypes.byref(a), ctypes.byref(b)))
    return a.value, b.value


def exported_symbols():
    """Names of every function declared in include/*.h."""
    names = []
    for f in sorted(os.listdir(HEADER_DIR)):
        if f.endswith(".h"):
            txt = open(os.path.join(HEADER_DIR, f)).read()
            names += re.findall(r"^\s*(?:const\s+)?[a-z_][\w\s\*]*?\b([a-z]\w*)\s*\(", txt, re.M)
    return sorted(set(n for n in names if not n.startswith(("if", "for", "while", "sizeof"))))


def library():
    return _lib


def last_error():
    return _lib.rexi_last_error().decode()


def coeffs(N, p0, Xc, phi=0):
    """Poles z_n and weights w_n of  psi_phi(x) ~ sum_n w_n / (z_n - x)  (complex128 arrays)."""
    z = np.empty(2 * N)
    w = np.empty(2 * N)
    _check(_lib.rexi_coeffs(int(N), float(p0), float(Xc), int(phi),
                            z.ctypes.data_as(_dp), w.ctypes.data_as(_dp)))
    return z.view(np.complex128), w.view(np.complex128)


def contour_select(X, N):
    p0 = ctypes.c_double()
    Xc = ctypes.c_double()
    _check(_lib.rexi_contour_select(float(X), int(N), ctypes.byref(p0), ctypes.byref(Xc)))
    return p0.value, Xc.value


def select_poles(z, w, X, precision="mixed", heavy_tau=-1.0, prune_tau=0.0, heavy_align=16):
    """(cls, pruned_gain): per pole 1 heavy, 0 light, -1 pruned, as a plan would classify them
    (host only)."""
    z = np.ascontiguousarray(np.asarray(z, dtype=np.complex128))
    w = np.ascontiguousarray(np.asarray(w, dtype=np.complex128))
    if z.shape != w.shape or z.ndim != 1:
        raise ValueError("z and w must be 1-D arrays of the same length")
    cls = np.empty(len(z), dtype=np.int32)
    pg = ctypes.c_double()
    _check(_lib.rexi_select_poles(_PREC[precision], len(z), z.ctypes.data_as(_dp), w.ctypes.data_as(_dp),
                                  float(X), float(heavy_tau), float(prune_tau), int(heavy_align),
                                  cls.ctypes.data_as(_ip), ctypes.byref(pg)))
    return cls, pg.value


def spectrum_bound(T, dt, omega, radius, phibar):
    return _lib.rexi_spectrum_bound(int(T), float(dt), float(omega), float(radius), float(phibar))


def nlm(T):
    return (T + 1) * (T + 2) // 2


def _stream_handle(stream):
    if stream is None:
        import torch
        return torch.cuda.current_stream().cuda_stream
    if isinstance(stream, int):
        return stream
    return stream.cuda_stream


class Plan:
    """REXI plan: U1 = sum_n w_n (z_n - dt L)^-1 U0 for batches of spectral states."""

    def __init__(self, T, N, dt, omega, radius, phibar, p0=None, Xc=None, z=None, w=None,
                 precision="fp64", heavy_tau=-1.0, max_batch=1, stream=None, prune_tau=0.0,
                 partition=None, fp64_tau=0.0):
        """partition: None, or (mode, rank, size) with mode "poles" or "m": this plan computes
        rank's share of the step (include/rexi.h part_mode); step_allreduce completes it."""
        d = PlanDesc()
        d.T, d.N, d.dt = int(T), int(N), float(dt)
        d.omega, d.radius, d.phibar = float(omega), float(radius), float(phibar)
        d.p0 = float(p0) if p0 is not None else 0.0
        d.Xc = float(Xc) if Xc is not None else 0.0
        self._zw = None
        if z is not None:
            zz = np.ascontiguousarray(np.asarray(z, dtype=np.complex128)).view(np.float64)
            ww = np.ascontiguousarray(np.asarray(w, dtype=np.complex128)).view(np.float64)
            self._zw = (zz, ww)
            d.z = zz.ctypes.data_as(_dp)
            d.w = ww.ctypes.data_as(_dp)
        d.precision = _PREC[precision] if isinstance(precision, str) else int(precision)
        d.heavy_tau = float(heavy_tau)
        d.max_batch = int(max_batch)
        d.stream = ctypes.c_void_p(_stream_handle(stream))
        d.prune_tau = float(prune_tau)
        d.fp64_tau = float(fp64_tau)
        if partition is not None:
            mode, rank, size = partition
            d.part_mode, d.part_rank, d.part_size = _PART[mode], int(rank), int(size)
        h = ctypes.c_void_p()
        _check(_lib.rexi_plan_create(ctypes.byref(d), ctypes.byref(h)))
        self._h = h
        self.T, self.N, self.nlm, self.max_batch = int(T), int(N), nlm(T), int(max_batch)

    def step(self, U0, U1, batch=None):
        """U0, U1: CUDA complex128 tensors of shape [batch, 3, nlm] (or [3, nlm])."""
        if batch is None:
            batch = 1 if U0.dim() == 2 else U0.shape[0]
        a0 = _dev_tensor(U0, batch * 3 * self.nlm, "complex128", "U0")
        a1 = _dev_tensor(U1, batch * 3 * self.nlm, "complex128", "U1")
        _check(_lib.rexi_step(self._h, a0, a1, int(batch)))
        return U1

    def step_raw(self, U0_ptr, U1_ptr, batch):
        return _lib.rexi_step(self._h, ctypes.c_void_p(U0_ptr), ctypes.c_void_p(U1_ptr), int(batch))

    def step_host(self, U0, U1=None):
        """Host numpy complex128 arrays [batch, 3, nlm]; copies inside the call."""
        U0 = np.ascontiguousarray(U0, dtype=np.complex128)
        batch = 1 if U0.ndim == 2 else U0.shape[0]
        if U1 is None:
            U1 = np.empty_like(U0)
        _check(_lib.rexi_step_host(self._h, U0.view(np.float64).ctypes.data_as(_dp),
                                   U1.view(np.float64).ctypes.data_as(_dp), int(batch)))
        return U1

    def step_host_ptr(self, U0_ptr, U1_ptr, batch):
        _check(_lib.rexi_step_host(self._h, ctypes.cast(U0_ptr, _dp), ctypes.cast(U1_ptr, _dp),
                                   int(batch)))

    def step_host_async_ptr(self, U0_ptr, U1_ptr, batch):
        """Pipelined host step (rexi_step_host_async): returns at once; U0 and U1 (page-locked
        host memory) must stay untouched until sync()."""
        _check(_lib.rexi_step_host_async(self._h, ctypes.cast(U0_ptr, _dp), ctypes.cast(U1_ptr, _dp),
                                         int(batch)))

    def sync(self):
        _check(_lib.rexi_sync(self._h))

    def info(self):
        i = PlanInfo()
        _check(_lib.rexi_plan_get_info(self._h, ctypes.byref(i)))
        return {k: getattr(i, k) for k, _ in PlanInfo._fields_}

    def poles(self):
        """(z, w, cls): the solved poles in internal order, then the pruned ones; cls is 1 for
        heavy, 0 for light and -1 for pruned poles."""
        z = np.empty(2 * self.N)
        w = np.empty(2 * self.N)
        hv = np.empty(self.N, dtype=np.int32)
        _check(_lib.rexi_plan_get_poles(self._h, z.ctypes.data_as(_dp), w.ctypes.data_as(_dp),
                                        hv.ctypes.data_as(_ip)))
        return z.view(np.complex128), w.view(np.complex128), hv

    def set_profiling(self, enable=True):
        _check(_lib.rexi_plan_set_profiling(self._h, 1 if enable else 0))

    def profile(self, reset=True):
        """{kernel name: (total ms, launches)} since the last reset (synchronises)."""
        ms = np.zeros(len(KERNEL_NAMES))
        n = np.zeros(len(KERNEL_NAMES), dtype=np.int32)
        _check(_lib.rexi_plan_get_profile(self._h, ms.ctypes.data_as(_dp), n.ctypes.data_as(_ip),
                                          1 if reset else 0))
        return {k: (float(ms[i]), int(n[i])) for i, k in enumerate(KERNEL_NAMES)}

    def close(self):
        if getattr(self, "_h", None) is not None and self._h.value:
            _lib.rexi_plan_destroy(self._h)
            self._h = ctypes.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


# ---- gravity-only REXI plans (include/rexi.h, rexi_lg_*) ---------------------------------
class LgDesc(ctypes.Structure):
    _fields_ = [("T", ctypes.c_int), ("N", ctypes.c_int), ("dt", ctypes.c_double),
                ("radius", ctypes.c_double), ("phibar", ctypes.c_double), ("p0", ctypes.c_double),
                ("Xc", ctypes.c_double), ("z", _dp), ("w", _dp), ("phi", ctypes.c_int),
                ("ident", ctypes.c_double), ("max_batch", ctypes.c_int), ("stream", ctypes.c_void_p)]


_lib.rexi_lg_create.argtypes = [ctypes.POINTER(LgDesc), ctypes.POINTER(ctypes.c_void_p)]
_lib.rexi_lg_destroy.argtypes = [ctypes.c_void_p]
_lib.rexi_lg_step.argtypes = [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int]
_lib.rexi_lg_sync.argtypes = [ctypes.c_void_p]
_lib.rexi_lg_get_operator.argtypes = [ctypes.c_void_p, _dp, _ip]


class LgPlan:
    """Gravity-only REXI plan: U1 = sum_p w_p (z_p - dt L_g)^-1 U0 (the lg_rexi_* methods)."""

    def __init__(self, T, N, dt, radius, phibar, p0=None, Xc=None, z=None, w=None, phi=0,
                 ident=0.0, max_batch=1, stream=None):
        d = LgDesc()
        d.T, d.N, d.dt = int(T), int(N), float(dt)
        d.radius, d.phibar = float(radius), float(phibar)
        d.p0 = float(p0) if p0 is not None else 0.0
        d.Xc = float(Xc) if Xc is not None else 0.0
        self._zw = None
        if z is not None:
            zz = np.ascontiguousarray(np.asarray(z, dtype=np.complex128)).view(np.float64)
            ww = np.ascontiguousarray(np.asarray(w, dtype=np.complex128)).view(np.float64)
            self._zw = (zz, ww)
            d.z = zz.ctypes.data_as(_dp)
            d.w = ww.ctypes.data_as(_dp)
        d.phi = int(phi)
        d.ident = float(ident)
        d.max_batch = int(max_batch)
        d.stream = ctypes.c_void_p(_stream_handle(stream))
        h = ctypes.c_void_p()
        _check(_lib.rexi_lg_create(ctypes.byref(d), ctypes.byref(h)))
        self._h = h
        self.T, self.N, self.nlm, self.max_batch = int(T), int(N), nlm(T), int(max_batch)

    def step(self, U0, U1, batch=None):
        """U0, U1: CUDA complex128 tensors [batch, 3, nlm] (or [3, nlm]); U1 may be U0."""
        if batch is None:
            batch = 1 if U0.dim() == 2 else U0.shape[0]
        a0 = _dev_tensor(U0, batch * 3 * self.nlm, "complex128", "U0")
        a1 = _dev_tensor(U1, batch * 3 * self.nlm, "complex128", "U1")
        _check(_lib.rexi_lg_step(self._h, a0, a1, int(batch)))
        return U1

    def step_raw(self, U0_ptr, U1_ptr, batch):
        return _lib.rexi_lg_step(self._h, ctypes.c_void_p(U0_ptr), ctypes.c_void_p(U1_ptr), int(batch))

    def sync(self):
        _check(_lib.rexi_lg_sync(self._h))

    def operator(self):
        """Per-degree pole sums [T+1, 4] complex (M_PhiPhi, M_PhiDelta, M_DeltaPhi, M_ZetaZeta)
        and whether the step applies their real parts."""
        M = np.empty(8 * (self.T + 1))
        r = ctypes.c_int()
        _check(_lib.rexi_lg_get_operator(self._h, M.ctypes.data_as(_dp), ctypes.byref(r)))
        return M.view(np.complex128).reshape(self.T + 1, 4), bool(r.value)

    def close(self):
        if getattr(self, "_h", None) is not None and self._h.value:
            _lib.rexi_lg_destroy(self._h)
            self._h = ctypes.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


# ---- spherical-harmonic transforms (include/sht.h) ------------------------------------
SH_FP64, SH_TF32, SH_BF16, SH_TF32X3, SH_DF = 0, 1, 2, 3, 4
_SH_PREC = {"fp64": SH_FP64, "tf32": SH_TF32, "bf16": SH_BF16, "tf32x3": SH_TF32X3, "df": SH_DF}


class ShDesc(ctypes.Structure):
    _fields_ = [("T", ctypes.c_int), ("nlat", ctypes.c_int), ("nlon", ctypes.c_int),
                ("radius", ctypes.c_double), ("precision", ctypes.c_int),
                ("max_fields", ctypes.c_int), ("stream", ctypes.c_void_p),
                ("epilogue_wait_polls", ctypes.c_int), ("polar_threshold", ctypes.c_double)]


class ShTableUse(ctypes.Structure):
    _fields_ = [("total", ctypes.c_longlong), ("needed_synth", ctypes.c_longlong),
                ("needed_anal", ctypes.c_longlong), ("streamed_synth", ctypes.c_longlong),
                ("streamed_anal", ctypes.c_longlong), ("threshold", ctypes.c_double)]


_lib.sh_plan_create.argtypes = [ctypes.POINTER(ShDesc), ctypes.POINTER(ctypes.c_void_p)]
_lib.sh_plan_destroy.argtypes = [ctypes.c_void_p]
_lib.sh_plan_get_grid.argtypes = [ctypes.c_void_p, _dp, _dp]
for _n in ("sh_synthesis", "sh_analysis"):
    getattr(_lib, _n).argtypes = [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int]
_lib.sh_plan_check.argtypes = [ctypes.c_void_p]
_lib.sh_plan_get_table_use.argtypes = [ctypes.c_void_p, ctypes.POINTER(ShTableUse)]
_lib.sh_plan_set_profiling.argtypes = [ctypes.c_void_p, ctypes.c_int]
_lib.sh_plan_get_profile.argtypes = [ctypes.c_void_p, _dp, _ip, ctypes.c_int]
SH_STAGE_NAMES = ("legendre_fp64", "legendre_df", "tc_gemm", "tc_epilogue", "fft")
for _n in ("sh_synthesis_uv", "sh_analysis_divcurl"):
    getattr(_lib, _n).argtypes = [ctypes.c_void_p] + [ctypes.c_void_p] * 4 + [ctypes.c_int]
_lib.sh_synthesis_mixed.argtypes = [ctypes.c_void_p] + [ctypes.c_void_p] * 2 + [ctypes.c_int] + \
    [ctypes.c_void_p] * 4 + [ctypes.c_int]
_lib.sh_analysis_mixed.argtypes = [ctypes.c_void_p] + [ctypes.c_void_p] * 4 + [ctypes.c_int] + \
    [ctypes.c_void_p] * 2 + [ctypes.c_int]


def _ptr(t):
    return ctypes.c_void_p(t.data_ptr())


class ShPlan:
    """Spherical-harmonic transforms on a Gauss grid (nlat x nlon), truncation T."""

    def __init__(self, T, nlat, nlon, radius, precision="fp64", max_fields=1, stream=None,
                 epilogue_wait_polls=0, polar_threshold=0.0):
        """polar_threshold: 0 = the library default (1e-19), > 0 = that threshold, < 0 = no
        polar truncation of the Legendre sums."""
        d = ShDesc()
        d.T, d.nlat, d.nlon, d.radius = int(T), int(nlat), int(nlon), float(radius)
        d.precision = _SH_PREC[precision] if isinstance(precision, str) else int(precision)
        d.max_fields = int(max_fields)
        d.stream = ctypes.c_void_p(_stream_handle(stream))
        d.epilogue_wait_polls = int(epilogue_wait_polls)
        d.polar_threshold = float(polar_threshold)
        h = ctypes.c_void_p()
        _check(_lib.sh_plan_create(ctypes.byref(d), ctypes.byref(h)))
        self._h = h
        self.T, self.nlat, self.nlon, self.nlm = int(T), int(nlat), int(nlon), nlm(T)

    def grid(self):
        mu = np.empty(self.nlat)
        w = np.empty(self.nlat)
        _check(_lib.sh_plan_get_grid(self._h, mu.ctypes.data_as(_dp), w.ctypes.data_as(_dp)))
        return mu, w

    def _spec(self, t, nfields, what):
        return _dev_tensor(t, int(nfields) * self.nlm, "complex128", what, at_least=True)

    def _grid(self, t, nfields, what):
        return _dev_tensor(t, int(nfields) * self.nlat * self.nlon, "float64", what, at_least=True)

    def synthesis(self, spec, grid, nfields=1):
        _check(_lib.sh_synthesis(self._h, self._spec(spec, nfields, "spec"),
                                 self._grid(grid, nfields, "grid"), int(nfields)))
        return grid

    def analysis(self, grid, spec, nfields=1):
        _check(_lib.sh_analysis(self._h, self._grid(grid, nfields, "grid"),
                                self._spec(spec, nfields, "spec"), int(nfields)))
        return spec

    def synthesis_uv(self, psi, chi, U, V, nfields=1):
        _check(_lib.sh_synthesis_uv(self._h, self._spec(psi, nfields, "psi"), self._spec(chi, nfields, "chi"),
                                    self._grid(U, nfields, "U"), self._grid(V, nfields, "V"), int(nfields)))
        return U, V

    def check(self):
        """Synchronise; raise if a device-side bounded wait gave up."""
        _check(_lib.sh_plan_check(self._h))

    def table_use(self):
        """Table entries per table: total, needed by the polar-truncated sums (synthesis,
        analysis), streamed by this plan's kernels, and the threshold in use (0: off)."""
        u = ShTableUse()
        _check(_lib.sh_plan_get_table_use(self._h, ctypes.byref(u)))
        return {k: getattr(u, k) for k, _ in ShTableUse._fields_}

    def set_profiling(self, enable=True):
        _check(_lib.sh_plan_set_profiling(self._h, 1 if enable else 0))

    def profile(self, reset=True):
        """{stage: (total ms, launches)} since the last reset (synchronises the stream)."""
        ms = np.zeros(len(SH_STAGE_NAMES))
        n = np.zeros(len(SH_STAGE_NAMES), dtype=np.int32)
        _check(_lib.sh_plan_get_profile(self._h, ms.ctypes.data_as(_dp), n.ctypes.data_as(_ip),
                                        1 if reset else 0))
        return {k: (float(ms[i]), int(n[i])) for i, k in enumerate(SH_STAGE_NAMES)}

    def analysis_divcurl(self, A, B, div, curl, nfields=1):
        _check(_lib.sh_analysis_divcurl(self._h, self._grid(A, nfields, "A"), self._grid(B, nfields, "B"),
                                        self._spec(div, nfields, "div"), self._spec(curl, nfields, "curl"),
                                        int(nfields)))
        return div, curl

    def synthesis_mixed(self, spec, grid, nfields, psi, chi, U, V, nvec):
        """Scalar synthesis of nfields spectra beside the velocity synthesis of nvec (psi,
        chi) pairs, in one pass (one read of each Legendre table)."""
        _check(_lib.sh_synthesis_mixed(self._h, self._spec(spec, nfields, "spec"), self._grid(grid, nfields, "grid"),
                                       int(nfields), self._spec(psi, nvec, "psi"), self._spec(chi, nvec, "chi"),
                                       self._grid(U, nvec, "U"), self._grid(V, nvec, "V"), int(nvec)))
        return grid, U, V

    def analysis_mixed(self, A, B, div, curl, nvec, grid, spec, nfields):
        """Divergence and curl of nvec vector fields beside the analysis of nfields scalar
        grids, in one pass."""
        _check(_lib.sh_analysis_mixed(self._h, self._grid(A, nvec, "A"), self._grid(B, nvec, "B"),
                                      self._spec(div, nvec, "div"), self._spec(curl, nvec, "curl"), int(nvec),
                                      self._grid(grid, nfields, "grid"), self._spec(spec, nfields, "spec"),
                                      int(nfields)))
        return div, curl, spec

    def close(self):
        if getattr(self, "_h", None) is not None and self._h.value:
            _lib.sh_plan_destroy(self._h)
            self._h = ctypes.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


# ---- nonlinear shallow-water step (include/swe.h) ---------------------------------------
SWE_VER1, SWE_VER0, SWE_ETDRK, SWE_IRK, SWE_LG_VER1, SWE_LG_ETDRK, SWE_LG_IRK_VER0 = range(7)
SWE_SCHEMES = {"ver1": SWE_VER1, "ver0": SWE_VER0, "etdrk": SWE_ETDRK, "irk": SWE_IRK,
               "lg_ver1": SWE_LG_VER1, "lg_etdrk": SWE_LG_ETDRK, "lg_irk_ver0": SWE_LG_IRK_VER0}


class SweDesc(ctypes.Structure):
    _fields_ = [("T", ctypes.c_int), ("nlat", ctypes.c_int), ("nlon", ctypes.c_int),
                ("dt", ctypes.c_double), ("omega", ctypes.c_double), ("radius", ctypes.c_double),
                ("phibar", ctypes.c_double), ("N", ctypes.c_int), ("p0", ctypes.c_double),
                ("Xc", ctypes.c_double), ("rexi_precision", ctypes.c_int),
                ("sh_precision", ctypes.c_int), ("scheme", ctypes.c_int),
                ("stream", ctypes.c_void_p), ("nsub", ctypes.c_int), ("visc", ctypes.c_double),
                ("visc_order", ctypes.c_int)]


_lib.swe_plan_create.argtypes = [ctypes.POINTER(SweDesc), ctypes.POINTER(ctypes.c_void_p)]
_lib.swe_plan_destroy.argtypes = [ctypes.c_void_p]
_lib.swe_step.argtypes = [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int]
_lib.swe_nonlinear.argtypes = [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p]
_lib.swe_plan_set_profiling.argtypes = [ctypes.c_void_p, ctypes.c_int]
_lib.swe_substeps.argtypes = [ctypes.c_int] + [ctypes.c_double] * 4


def swe_substeps(T, tau, umax, radius, courant=1.0):
    """Explicit midpoint sub-steps over tau so that the advective phase change of degree T under
    the wind umax stays within `courant` radians per sub-step (include/swe.h)."""
    n = _lib.swe_substeps(int(T), float(tau), float(umax), float(radius), float(courant))
    return _check(n) if n < 0 else int(n)
_lib.swe_plan_get_profile.argtypes = [ctypes.c_void_p, _dp, _ip, ctypes.c_int]
SWE_STAGE_NAMES = ("rexi", "legendre", "fft", "grid_products")


class SwePlan:
    """Nonlinear SWE step on a Gauss grid: Strang split (l_rexi_n_erk_ver1 / ver0), ETD2RK
    (l_rexi_n_etdrk), Crank-Nicolson in the Strang split (l_irk_n_erk_ver1), or the Coriolis
    term in the explicit part (lg_rexi_lc_n_erk_ver1 "lg_ver1", lg_rexi_lc_n_etdrk "lg_etdrk",
    lg_irk_lc_n_erk_ver0 "lg_irk_ver0")."""

    def __init__(self, T, nlat, nlon, dt, omega, radius, phibar, N, p0, Xc, rexi_precision="fp64",
                 sh_precision="fp64", scheme="ver1", stream=None, nsub=1, visc=0.0, visc_order=2):
        d = SweDesc()
        d.T, d.nlat, d.nlon, d.dt = int(T), int(nlat), int(nlon), float(dt)
        d.omega, d.radius, d.phibar = float(omega), float(radius), float(phibar)
        d.N, d.p0, d.Xc = int(N), float(p0), float(Xc)
        d.rexi_precision = _PREC[rexi_precision] if isinstance(rexi_precision, str) else int(rexi_precision)
        d.sh_precision = _SH_PREC[sh_precision] if isinstance(sh_precision, str) else int(sh_precision)
        d.scheme = SWE_SCHEMES[scheme] if isinstance(scheme, str) else int(scheme)
        d.stream = ctypes.c_void_p(_stream_handle(stream))
        d.nsub = int(nsub)
        d.visc, d.visc_order = float(visc), int(visc_order)
        h = ctypes.c_void_p()
        _check(_lib.swe_plan_create(ctypes.byref(d), ctypes.byref(h)))
        self._h = h
        self.T, self.nlm = int(T), nlm(T)

    def step(self, state, nsteps=1):
        _check(_lib.swe_step(self._h, _dev_tensor(state, 3 * self.nlm, "complex128", "state"), int(nsteps)))
        return state

    def nonlinear(self, state, tendency):
        _check(_lib.swe_nonlinear(self._h, _dev_tensor(state, 3 * self.nlm, "complex128", "state"),
                                  _dev_tensor(tendency, 3 * self.nlm, "complex128", "tendency")))
        return tendency

    def set_profiling(self, enable=True):
        _check(_lib.swe_plan_set_profiling(self._h, 1 if enable else 0))

    def profile(self, reset=True):
        """{stage: (total ms, launches)} since the last reset (synchronises the stream)."""
        ms = np.zeros(len(SWE_STAGE_NAMES))
        n = np.zeros(len(SWE_STAGE_NAMES), dtype=np.int32)
        _check(_lib.swe_plan_get_profile(self._h, ms.ctypes.data_as(_dp), n.ctypes.data_as(_ip),
                                         1 if reset else 0))
        return {k: (float(ms[i]), int(n[i])) for i, k in enumerate(SWE_STAGE_NAMES)}

    def close(self):
        if getattr(self, "_h", None) is not None and self._h.value:
            _lib.swe_plan_destroy(self._h)
            self._h = ctypes.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
