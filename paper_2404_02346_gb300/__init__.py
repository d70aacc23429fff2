"""GB300 wave lattice Boltzmann acoustic-radiation-force library: Python binding.

Argument marshalling only.  Every step of the computation runs in the CUDA
library ``_build/libwlb.so`` behind the C ABI of ``include/wlb.h``; PyTorch
supplies the device workspace and the CUDA stream.  There is no CPU path: if
the library has not been built, importing the binding's entry points raises.

Names follow ``include/wlb.h``: ``Solver.init/step/force/run/fields/surface/
mask/info`` wrap ``wlb_init/wlb_step/...``.
"""
import ctypes
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "_build", "libwlb.so")

WLB_OK, WLB_ERR_ARG, WLB_ERR_UNSTABLE, WLB_ERR_CUDA, WLB_ERR_OOM, WLB_ERR_STATE, WLB_ERR_TIMEOUT = range(7)
WLB_D2Q5, WLB_D3Q7 = 0, 1
WLB_POP_F32, WLB_POP_F64, WLB_POP_F16 = 0, 1, 2


class WlbError(RuntimeError):
    def __init__(self, status, msg):
        super().__init__(msg)
        self.status = status


class Params(ctypes.Structure):
    """Mirror of ``wlb_params``."""
    _fields_ = [
        ("lattice", ctypes.c_int),
        ("nx", ctypes.c_int), ("ny", ctypes.c_int), ("nz", ctypes.c_int),
        ("wave_axis", ctypes.c_int),
        ("c0", ctypes.c_double), ("cp", ctypes.c_double), ("rho0", ctypes.c_double),
        ("p_a", ctypes.c_double), ("wavelength", ctypes.c_double), ("antinode", ctypes.c_double),
        ("center", ctypes.c_double * 3),
        ("radius", ctypes.c_double), ("interface_d", ctypes.c_double),
        ("surface_radius", ctypes.c_double),
        ("n_surface", ctypes.c_int),
        ("n_periods", ctypes.c_int), ("n_avg_periods", ctypes.c_int),
        ("precision", ctypes.c_int),
        ("boundary", ctypes.c_int),
        ("wall_damping", ctypes.c_double), ("source_amplitude", ctypes.c_double),
    ]


class Info(ctypes.Structure):
    """Mirror of ``wlb_info``."""
    _fields_ = [
        ("dim", ctypes.c_int), ("q", ctypes.c_int),
        ("cells", ctypes.c_longlong), ("period", ctypes.c_longlong),
        ("n_steps", ctypes.c_longlong), ("n_window", ctypes.c_longlong),
        ("steps_done", ctypes.c_longlong), ("samples_done", ctypes.c_longlong),
        ("bytes_per_update", ctypes.c_double), ("vector_path", ctypes.c_int),
        ("steps_per_launch", ctypes.c_int),
        ("two_step_rows", ctypes.c_int),
        ("two_step_segments", ctypes.c_int),
        ("two_step_tiles", ctypes.c_int),
        ("two_step_staging_warp", ctypes.c_int),
        ("two_step_c2_staged", ctypes.c_int),
    ]


class BatchTuning(ctypes.Structure):
    """Mirror of ``wlb_batch_tuning``."""
    _fields_ = [("threads_per_block", ctypes.c_int), ("blocks_per_sm", ctypes.c_int),
                ("ms_per_step", ctypes.c_float), ("z_chunk", ctypes.c_int), ("slab_rows_cap", ctypes.c_int),
                ("one_chunk_per_lane", ctypes.c_int), ("plans_tried", ctypes.c_int),
                ("staging_warp", ctypes.c_int)]


class BatchInfo(ctypes.Structure):
    """Mirror of ``wlb_batch_info``."""
    _fields_ = [("count", ctypes.c_int), ("total_rows", ctypes.c_longlong),
                ("total_points", ctypes.c_longlong), ("max_steps", ctypes.c_longlong),
                ("lattice_updates", ctypes.c_longlong), ("threads_per_block", ctypes.c_int),
                ("blocks_per_sm", ctypes.c_int), ("row_chunks", ctypes.c_int),
                ("steps_per_launch", ctypes.c_int), ("total_ctas", ctypes.c_int)]


_lib = None
# Functions declared in include/wlb.h, with their ctypes signatures.
_VP = ctypes.c_void_p
_DP = ctypes.POINTER(ctypes.c_double)
_SIGNATURES = {
    "wlb_validate": (ctypes.c_int, [ctypes.POINTER(Params)]),
    "wlb_workspace_bytes": (ctypes.c_int, [ctypes.POINTER(Params), ctypes.POINTER(ctypes.c_size_t)]),
    "wlb_create": (ctypes.c_int, [ctypes.POINTER(Params), _VP, ctypes.c_size_t, _VP, ctypes.POINTER(_VP)]),
    "wlb_init": (ctypes.c_int, [_VP]),
    "wlb_step": (ctypes.c_int, [_VP, ctypes.c_longlong, ctypes.c_int]),
    "wlb_force": (ctypes.c_int, [_VP, _DP]),
    "wlb_run": (ctypes.c_int, [_VP, _DP]),
    "wlb_fields": (ctypes.c_int, [_VP, _DP, _DP]),
    "wlb_surface": (ctypes.c_int, [_VP, _DP]),
    "wlb_mask": (ctypes.c_int, [_VP, ctypes.POINTER(ctypes.c_ubyte)]),
    "wlb_state_bytes": (ctypes.c_int, [_VP, ctypes.POINTER(ctypes.c_size_t)]),
    "wlb_set_deadline": (ctypes.c_int, [_VP, ctypes.c_double]),
    "wlb_force_history": (ctypes.c_int, [_VP, ctypes.POINTER(ctypes.c_double),
                                         ctypes.POINTER(ctypes.c_longlong), ctypes.c_int,
                                         ctypes.POINTER(ctypes.c_int)]),
    "wlb_save_state": (ctypes.c_int, [_VP, _VP, ctypes.c_size_t]),
    "wlb_load_state": (ctypes.c_int, [_VP, _VP, ctypes.c_size_t]),
    "wlb_get_info": (ctypes.c_int, [_VP, ctypes.POINTER(Info)]),
    "wlb_set_two_step": (ctypes.c_int, [_VP, ctypes.c_int, ctypes.c_int]),
    "wlb_set_two_step_tiles": (ctypes.c_int, [_VP, ctypes.c_int]),
    "wlb_set_two_step_staging": (ctypes.c_int, [_VP, ctypes.c_int]),
    "wlb_set_two_step_c2": (ctypes.c_int, [_VP, ctypes.c_int]),
    "wlb_destroy": (ctypes.c_int, [_VP]),
    "wlb_average_noalloc": (ctypes.c_int, [_VP, ctypes.c_longlong, _DP]),
    "wlb_batch_workspace_bytes": (ctypes.c_int, [ctypes.POINTER(Params), ctypes.c_int,
                                                 ctypes.POINTER(ctypes.c_size_t)]),
    "wlb_batch_create": (ctypes.c_int, [ctypes.POINTER(Params), ctypes.c_int, _VP, ctypes.c_size_t, _VP,
                                        ctypes.POINTER(_VP)]),
    "wlb_batch_autotune": (ctypes.c_int, [_VP, ctypes.c_int, ctypes.POINTER(BatchTuning)]),
    "wlb_batch_run": (ctypes.c_int, [_VP, _DP]),
    "wlb_batch_get_info": (ctypes.c_int, [_VP, ctypes.POINTER(BatchInfo)]),
    "wlb_batch_set_two_step": (ctypes.c_int, [_VP, ctypes.c_int]),
    "wlb_batch_last_error": (ctypes.c_char_p, [_VP]),
    "wlb_batch_destroy": (ctypes.c_int, [_VP]),
    "wlb_mlp_param_count": (ctypes.c_int, []),
    "wlb_mlp_create": (ctypes.c_int, [ctypes.c_int, ctypes.POINTER(ctypes.c_float), ctypes.POINTER(ctypes.c_float),
                                      _VP, ctypes.POINTER(_VP)]),
    "wlb_mlp_init_weights": (ctypes.c_int, [_VP, ctypes.c_ulonglong]),
    "wlb_mlp_set_weights": (ctypes.c_int, [_VP, ctypes.POINTER(ctypes.c_float)]),
    "wlb_mlp_get_weights": (ctypes.c_int, [_VP, ctypes.POINTER(ctypes.c_float)]),
    "wlb_mlp_loss_grad": (ctypes.c_int, [_VP, _VP, _VP, ctypes.c_int, ctypes.POINTER(ctypes.c_float),
                                         ctypes.POINTER(ctypes.c_float)]),
    "wlb_mlp_train": (ctypes.c_int, [_VP, _VP, _VP, ctypes.c_longlong, ctypes.c_int, ctypes.c_int, ctypes.c_float,
                                     ctypes.c_float, ctypes.c_ulonglong, ctypes.POINTER(ctypes.c_float)]),
    "wlb_mlp_predict": (ctypes.c_int, [_VP, _VP, ctypes.c_longlong, _VP, _VP]),
    "wlb_mlp_set_fused": (ctypes.c_int, [_VP, ctypes.c_int]),
    "wlb_mlp_last_error": (ctypes.c_char_p, [_VP]),
    "wlb_mlp_destroy": (ctypes.c_int, [_VP]),
    "wlb_status_str": (ctypes.c_char_p, [ctypes.c_int]),
    "wlb_last_error": (ctypes.c_char_p, [_VP]),
}


def lib():
    """Load the CUDA library (raises if it has not been built)."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise ImportError("CUDA library not built: %s (run __graft_entry__.build())" % LIB_PATH)
        L = ctypes.CDLL(LIB_PATH)
        for name, (res, args) in _SIGNATURES.items():
            fn = getattr(L, name)
            fn.restype = res
            fn.argtypes = args
        _lib = L
    return _lib


def _check(status, handle=None, what=""):
    if status != WLB_OK:
        L = lib()
        detail = L.wlb_last_error(handle).decode() if handle else ""
        raise WlbError(status, "%s: %s %s" % (what, L.wlb_status_str(status).decode(), detail))


def params_from_problem(prob, precision=None):
    """wlb_params from a problem dictionary (see workloads.py)."""
    p = Params()
    dim = int(prob["dim"])
    p.lattice = WLB_D2Q5 if dim == 2 else WLB_D3Q7
    n = list(prob["n"]) + [1] * (3 - len(prob["n"]))
    p.nx, p.ny, p.nz = (int(v) for v in n[:3])
    p.wave_axis = int(prob["wave_axis"])
    for k in ("c0", "cp", "rho0", "p_a", "wavelength", "antinode", "radius", "interface_d",
              "surface_radius"):
        setattr(p, k, float(prob[k]))
    c = list(prob["center"]) + [0.0] * (3 - len(prob["center"]))
    for a in range(3):
        p.center[a] = float(c[a])
    p.n_surface = int(prob["n_surface"])
    T = prob["period"] if "period" in prob else int(round(prob["wavelength"] / prob["c0"]))
    if prob["n_steps"] % T or prob["n_window"] % T:
        raise ValueError("n_steps and n_window must be whole periods")
    p.n_periods = int(prob["n_steps"] // T)
    p.n_avg_periods = int(prob["n_window"] // T)
    prec = precision or prob.get("precision", "f32")
    p.precision = {"f32": WLB_POP_F32, "f64": WLB_POP_F64, "f16": WLB_POP_F16}[prec]
    p.boundary = 1 if prob.get("boundary", "periodic") == "driven" else 0
    p.wall_damping = float(prob.get("wall_damping", 0.99))
    p.source_amplitude = float(prob.get("source_amplitude", 0.0))
    return p


def workspace_bytes(params):
    nb = ctypes.c_size_t()
    _check(lib().wlb_workspace_bytes(ctypes.byref(params), ctypes.byref(nb)), what="wlb_workspace_bytes")
    return nb.value


def validate(params):
    return lib().wlb_validate(ctypes.byref(params))


class Solver:
    """One lattice problem on the current CUDA device.

    Device memory is one torch uint8 tensor handed to ``wlb_create``; work is
    issued on ``stream`` (a torch.cuda.Stream; default: the current stream).
    """

    def __init__(self, problem, stream=None, precision=None):
        import torch  # device memory and streams only

        self.problem = problem
        self.params = params_from_problem(problem, precision)
        L = lib()
        nb = workspace_bytes(self.params)
        self.stream = stream if stream is not None else torch.cuda.current_stream()
        self._ws = torch.empty(nb, dtype=torch.uint8, device=self.stream.device)
        h = _VP()
        _check(L.wlb_create(ctypes.byref(self.params), ctypes.c_void_p(self._ws.data_ptr()), nb,
                            ctypes.c_void_p(self.stream.cuda_stream), ctypes.byref(h)), what="wlb_create")
        self._h = h
        info = self.info()
        self.dim, self.q, self.cells = info.dim, info.q, info.cells
        self.shape = (self.params.nz, self.params.ny, self.params.nx)

    # -- lifetime --------------------------------------------------------
    def close(self):
        if getattr(self, "_h", None):
            lib().wlb_destroy(self._h)
            self._h = None
            self._ws = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    # -- calls -----------------------------------------------------------
    def info(self):
        out = Info()
        _check(lib().wlb_get_info(self._h, ctypes.byref(out)), self._h, "wlb_get_info")
        return out

    def init(self):
        _check(lib().wlb_init(self._h), self._h, "wlb_init")

    def set_two_step(self, enable=True, slab_rows=0, chunks_per_lane=0):
        """Steps two per launch (wlb_set_two_step); chunks_per_lane 0 lets the
        library choose, 1 or 2 asks for that lane layout."""
        mode = (1 + int(chunks_per_lane)) if enable else 0
        _check(lib().wlb_set_two_step(self._h, mode, int(slab_rows)), self._h, "wlb_set_two_step")

    def set_two_step_tiles(self, tiles=0):
        """x-tiles per row of the two-step kernel (wlb_set_two_step_tiles): 0
        lets the library choose, 1 keeps whole rows, n splits rows in n."""
        _check(lib().wlb_set_two_step_tiles(self._h, int(tiles)), self._h, "wlb_set_two_step_tiles")

    def set_two_step_staging(self, staging=0):
        """Who stages the two-step kernel's planes (wlb_set_two_step_staging):
        0 automatic, 1 warp 0, 2 a dedicated warp."""
        _check(lib().wlb_set_two_step_staging(self._h, int(staging)), self._h, "wlb_set_two_step_staging")

    def set_two_step_c2(self, c2=0):
        """Where the two-step kernel reads band rows' c^2 (wlb_set_two_step_c2):
        0 automatic, 1 staged in shared memory, 2 from L2."""
        _check(lib().wlb_set_two_step_c2(self._h, int(c2)), self._h, "wlb_set_two_step_c2")

    def step(self, n, sample=False):
        _check(lib().wlb_step(self._h, int(n), 1 if sample else 0), self._h, "wlb_step")

    def set_deadline(self, seconds):
        """Host-clock limit of run() (wlb_set_deadline); 0 turns it off."""
        _check(lib().wlb_set_deadline(self._h, float(seconds)), self._h, "wlb_set_deadline")

    def force(self):
        F = np.zeros(3)
        _check(lib().wlb_force(self._h, F.ctypes.data_as(_DP)), self._h, "wlb_force")
        return F

    def run(self):
        F = np.zeros(3)
        _check(lib().wlb_run(self._h, F.ctypes.data_as(_DP)), self._h, "wlb_run")
        return F

    def fields(self):
        p1 = np.zeros(self.shape)
        u1 = np.zeros((self.dim,) + self.shape)
        _check(lib().wlb_fields(self._h, p1.ctypes.data_as(_DP), u1.ctypes.data_as(_DP)), self._h,
               "wlb_fields")
        return p1, u1

    def surface(self):
        pts = np.zeros((max(self.params.n_surface, 1), 7))
        _check(lib().wlb_surface(self._h, pts.ctypes.data_as(_DP)), self._h, "wlb_surface")
        return pts[: self.params.n_surface]

    def mask(self):
        m = np.zeros(self.shape, dtype=np.uint8)
        _check(lib().wlb_mask(self._h, m.ctypes.data_as(ctypes.POINTER(ctypes.c_ubyte))), self._h,
               "wlb_mask")
        return m

    def force_history(self, with_samples=False):
        """Force of every recorded fold (each full sampled period, and a partial
        one folded by force()), (count, 3); with_samples also returns the sample
        count of each row (wlb_force_history)."""
        cap = max(int(self.params.n_periods), 1) + 1
        out = np.zeros((cap, 3))
        smp = np.zeros(cap, dtype=np.int64)
        n = ctypes.c_int()
        _check(lib().wlb_force_history(self._h, out.ctypes.data_as(_DP),
                                       smp.ctypes.data_as(ctypes.POINTER(ctypes.c_longlong)), cap,
                                       ctypes.byref(n)), self._h, "wlb_force_history")
        k = min(n.value, cap)
        return (out[:k], smp[:k]) if with_samples else out[:k]

    def save_state(self):
        """Checkpoint (wlb_save_state) as a numpy uint8 array."""
        n = ctypes.c_size_t()
        _check(lib().wlb_state_bytes(self._h, ctypes.byref(n)), self._h, "wlb_state_bytes")
        buf = np.empty(n.value, dtype=np.uint8)
        _check(lib().wlb_save_state(self._h, ctypes.c_void_p(buf.ctypes.data), n.value), self._h,
               "wlb_save_state")
        return buf

    def load_state(self, buf):
        """Resume from a checkpoint written by save_state (wlb_load_state)."""
        buf = np.ascontiguousarray(buf, dtype=np.uint8)
        _check(lib().wlb_load_state(self._h, ctypes.c_void_p(buf.ctypes.data), buf.size), self._h,
               "wlb_load_state")


def compute_force(problem, precision=None):
    """One force evaluation through the public API (host in, host out)."""
    with Solver(problem, precision=precision) as s:
        return s.run()


class Batch:
    """Many independent lattices (same lattice type and precision) stepped
    together by the batched kernels (wlb_batch_*).  One torch workspace."""

    def __init__(self, problems, stream=None, precision=None):
        import torch

        self.problems = list(problems)
        n = len(self.problems)
        arr = (Params * n)(*[params_from_problem(p, precision) for p in self.problems])
        self._params = arr
        L = lib()
        nb = ctypes.c_size_t()
        _check(L.wlb_batch_workspace_bytes(arr, n, ctypes.byref(nb)), what="wlb_batch_workspace_bytes")
        self.stream = stream if stream is not None else torch.cuda.current_stream()
        self._ws = torch.empty(nb.value, dtype=torch.uint8, device=self.stream.device)
        h = _VP()
        _check(L.wlb_batch_create(arr, n, ctypes.c_void_p(self._ws.data_ptr()), nb.value,
                                  ctypes.c_void_p(self.stream.cuda_stream), ctypes.byref(h)),
               what="wlb_batch_create")
        self._h = h
        self.count = n

    def _bcheck(self, status, what):
        if status != WLB_OK:
            L = lib()
            raise WlbError(status, "%s: %s %s" % (what, L.wlb_status_str(status).decode(),
                                                   L.wlb_batch_last_error(self._h).decode()))

    def info(self):
        out = BatchInfo()
        self._bcheck(lib().wlb_batch_get_info(self._h, ctypes.byref(out)), "wlb_batch_get_info")
        return out

    def set_two_step(self, enable=True):
        """Two steps per launch for the whole batch (wlb_batch_set_two_step)."""
        self._bcheck(lib().wlb_batch_set_two_step(self._h, 1 if enable else 0), "wlb_batch_set_two_step")

    def autotune(self, steps_per_trial=16):
        t = BatchTuning()
        self._bcheck(lib().wlb_batch_autotune(self._h, int(steps_per_trial), ctypes.byref(t)),
                     "wlb_batch_autotune")
        return {"threads_per_block": t.threads_per_block, "blocks_per_sm": t.blocks_per_sm,
                "ms_per_step": t.ms_per_step, "z_chunk": t.z_chunk, "slab_rows_cap": t.slab_rows_cap,
                "one_chunk_per_lane": t.one_chunk_per_lane, "plans_tried": t.plans_tried,
                "staging_warp": t.staging_warp}

    def run(self):
        F = np.zeros((self.count, 3))
        self._bcheck(lib().wlb_batch_run(self._h, F.ctypes.data_as(_DP)), "wlb_batch_run")
        return F

    def close(self):
        if getattr(self, "_h", None):
            lib().wlb_batch_destroy(self._h)
            self._h = None
            self._ws = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()


_FP = ctypes.POINTER(ctypes.c_float)


class MLP:
    """The surrogate network (wlb_mlp_*).  Samples and outputs are torch CUDA
    tensors (float32); weights and gradients come back as numpy float32."""

    def __init__(self, x_lo, x_hi, batch_max=4096, stream=None):
        import torch

        self.stream = stream if stream is not None else torch.cuda.current_stream()
        lo = (ctypes.c_float * 4)(*[float(v) for v in x_lo])
        hi = (ctypes.c_float * 4)(*[float(v) for v in x_hi])
        h = _VP()
        _check(lib().wlb_mlp_create(int(batch_max), lo, hi, ctypes.c_void_p(self.stream.cuda_stream),
                                    ctypes.byref(h)), what="wlb_mlp_create")
        self._h = h
        self.n_params = lib().wlb_mlp_param_count()
        self.batch_max = batch_max

    def _mcheck(self, status, what):
        if status != WLB_OK:
            L = lib()
            raise WlbError(status, "%s: %s %s" % (what, L.wlb_status_str(status).decode(),
                                                   L.wlb_mlp_last_error(self._h).decode()))

    def init_weights(self, seed):
        self._mcheck(lib().wlb_mlp_init_weights(self._h, int(seed)), "wlb_mlp_init_weights")

    def set_weights(self, w):
        w = np.ascontiguousarray(w, dtype=np.float32)
        self._mcheck(lib().wlb_mlp_set_weights(self._h, w.ctypes.data_as(_FP)), "wlb_mlp_set_weights")

    def get_weights(self):
        w = np.zeros(self.n_params, dtype=np.float32)
        self._mcheck(lib().wlb_mlp_get_weights(self._h, w.ctypes.data_as(_FP)), "wlb_mlp_get_weights")
        return w

    def loss_grad(self, x, t):
        loss = ctypes.c_float()
        g = np.zeros(self.n_params, dtype=np.float32)
        self._mcheck(lib().wlb_mlp_loss_grad(self._h, ctypes.c_void_p(x.data_ptr()), ctypes.c_void_p(t.data_ptr()),
                                             int(x.shape[0]), ctypes.byref(loss), g.ctypes.data_as(_FP)),
                     "wlb_mlp_loss_grad")
        return loss.value, g

    def train(self, x, t, epochs, batch=512, lr=1e-3, lr_final=5e-5, seed=1):
        hist = np.zeros(epochs, dtype=np.float32)
        self._mcheck(lib().wlb_mlp_train(self._h, ctypes.c_void_p(x.data_ptr()), ctypes.c_void_p(t.data_ptr()),
                                         int(x.shape[0]), int(epochs), int(batch), float(lr), float(lr_final),
                                         int(seed), hist.ctypes.data_as(_FP)), "wlb_mlp_train")
        return hist

    def set_fused(self, fused):
        """True (default): predict with the one-launch fused network; False:
        one GEMM launch per layer (the training forward)."""
        self._mcheck(lib().wlb_mlp_set_fused(self._h, 1 if fused else 0), "wlb_mlp_set_fused")

    def predict(self, x):
        import torch

        n = int(x.shape[0])
        y = torch.empty(n, dtype=torch.float32, device=x.device)
        inside = torch.empty(n, dtype=torch.uint8, device=x.device)
        self._mcheck(lib().wlb_mlp_predict(self._h, ctypes.c_void_p(x.data_ptr()), n, ctypes.c_void_p(y.data_ptr()),
                                           ctypes.c_void_p(inside.data_ptr())), "wlb_mlp_predict")
        return y, inside

    def close(self):
        if getattr(self, "_h", None):
            lib().wlb_mlp_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
