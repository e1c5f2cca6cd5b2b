"""ctypes binding of libhdd.so (argument marshalling only).

Every step of the likelihood path runs in the library's CUDA kernels; this module
only converts Python / PyTorch arguments into the plain pointers and sizes of the
C ABI declared in include/hdd.h.  PyTorch provides device memory and streams.
There is no CPU fallback: if the library cannot be loaded, every call raises.
"""
from __future__ import annotations

import ctypes as C
import os

import numpy as np

_PKG = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_PKG, "_build", "libhdd.so")

HDD_OK, HDD_EINVAL, HDD_ENOMEM, HDD_ECUDA, HDD_ENOTSPD, HDD_ENOCONV, HDD_ETIMEOUT, HDD_ESTATE = 0, -1, -2, -3, -4, -5, -6, -7
HDD_FP64, HDD_MIXED_FP32 = 0, 1
HDD_OBS_VERTEX, HDD_OBS_MEANS = 0, 1

EXPORTED = [
    "hdd_plan", "hdd_plan_destroy", "hdd_workspace_size", "hdd_assemble", "hdd_upsweep",
    "hdd_point_solve", "hdd_loglik", "hdd_evaluate_host", "hdd_plan_info", "hdd_node_info",
    "hdd_node_indices", "hdd_status_string", "hdd_last_error", "hdd_evaluate_static",
    "hdd_profile_begin", "hdd_profile_end", "hdd_kappa", "hdd_solve_loads", "hdd_subdomain_means",
    "hdd_set_wait_bound", "hdd_mean_functionals", "hdd_multi_create", "hdd_multi_destroy", "hdd_multi_upsweep",
    "hdd_multi_evaluate", "hdd_multi_info", "hdd_data_scratch_size", "hdd_solve_data", "hdd_set_sweep_fusion",
    "hdd_multi_capture", "hdd_graph_launch", "hdd_graph_destroy",
]
STATIC_WORKSPACE_BYTES = 32 << 20


class PlanDesc(C.Structure):
    _fields_ = [
        ("N", C.c_int32), ("leaf", C.c_int32), ("n_z", C.c_int32),
        ("kl_basis", C.POINTER(C.c_double)), ("f", C.c_double),
        ("n_obs", C.c_int32), ("obs_vertex", C.POINTER(C.c_int32)),
        ("sigma", C.c_double), ("precision", C.c_int32), ("ir_max_iter", C.c_int32),
        ("ir_tol", C.c_double), ("fp64_top_levels", C.c_int32), ("fuse_height", C.c_int32),
        ("device", C.c_int32), ("obs_kind", C.c_int32),
    ]


class PlanInfo(C.Structure):
    _fields_ = [
        ("n_nodes", C.c_int32), ("n_leaves", C.c_int32), ("depth", C.c_int32), ("height", C.c_int32),
        ("n_visited", C.c_int32), ("max_front", C.c_int32),
        ("flops_upsweep", C.c_double), ("flops_point_solve", C.c_double),
        ("factor_bytes", C.c_double), ("schur_bytes", C.c_double),
        ("launches_upsweep", C.c_int32), ("launches_evaluate", C.c_int32),
        ("bytes_upsweep_tiny", C.c_double), ("bytes_upsweep_small", C.c_double),
        ("bytes_upsweep_large", C.c_double),
        ("bytes_upsweep_fused", C.c_double), ("bytes_forward", C.c_double),
        ("bytes_descent_all", C.c_double), ("bytes_descent_visited", C.c_double),
        ("bytes_residual", C.c_double), ("bytes_assemble", C.c_double), ("bytes_kl_basis", C.c_double),
        ("bytes_upsweep_leaf", C.c_double), ("n_condensed_leaves", C.c_int32),
        ("sweep_fuse_height", C.c_int32),
    ]


class KernelStat(C.Structure):
    _fields_ = [("name", C.c_char * 24), ("launches", C.c_int32), ("ms", C.c_double), ("flops", C.c_double)]


class NodeInfo(C.Structure):
    _fields_ = [(n, C.c_int32) for n in
                ("x0", "x1", "y0", "y1", "parent", "child0", "child1", "depth", "height", "m", "b", "visited")]


_lib = None


def load_library() -> C.CDLL:
    """Load libhdd.so (built by paper_1708_02207_gb300.build); raises if it is missing."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(LIB_PATH):
        raise RuntimeError(f"{LIB_PATH} is missing: run paper_1708_02207_gb300.build.build() first "
                           "(the HDD path has no CPU fallback)")
    lib = C.CDLL(LIB_PATH)
    vp, i32, pd, pi32 = C.c_void_p, C.c_int32, C.POINTER(C.c_double), C.POINTER(C.c_int32)
    lib.hdd_plan.argtypes = [C.POINTER(PlanDesc), C.POINTER(vp)]
    lib.hdd_plan_destroy.argtypes = [vp]
    lib.hdd_workspace_size.argtypes = [vp, i32, C.POINTER(C.c_size_t)]
    lib.hdd_assemble.argtypes = [vp, vp, i32, vp, vp]
    lib.hdd_upsweep.argtypes = [vp, i32, vp, vp]
    lib.hdd_point_solve.argtypes = [vp, i32, vp, vp, vp]
    lib.hdd_loglik.argtypes = [vp, i32, vp, vp, vp, i32, vp, vp, vp]
    lib.hdd_evaluate_host.argtypes = [vp, i32, vp, pd, pd, i32, pd, pd, pi32, vp]
    lib.hdd_evaluate_static.argtypes = [vp, i32, vp, vp, i32, vp, vp, vp, vp]
    lib.hdd_kappa.argtypes = [vp, i32, vp, vp, vp]
    lib.hdd_solve_loads.argtypes = [vp, i32, vp, vp, i32, vp, vp, vp]
    lib.hdd_subdomain_means.argtypes = [vp, i32, vp, C.c_int64, vp, vp]
    lib.hdd_set_wait_bound.argtypes = [vp, C.c_uint32, i32, i32]
    lib.hdd_set_sweep_fusion.argtypes = [vp, i32]
    lib.hdd_mean_functionals.argtypes = [vp, i32, vp, vp, vp, vp]
    lib.hdd_multi_create.argtypes = [C.POINTER(vp), i32, pi32, C.POINTER(vp), C.POINTER(vp)]
    lib.hdd_multi_destroy.argtypes = [vp]
    lib.hdd_multi_capture.argtypes = [vp, C.POINTER(vp), C.POINTER(vp), pi32, C.POINTER(vp), C.POINTER(vp),
                                      C.POINTER(vp), C.POINTER(vp)]
    lib.hdd_graph_launch.argtypes = [vp, vp]
    lib.hdd_graph_destroy.argtypes = [vp]
    lib.hdd_multi_upsweep.argtypes = [vp, vp]
    lib.hdd_multi_evaluate.argtypes = [vp, C.POINTER(vp), C.POINTER(vp), pi32, C.POINTER(vp), C.POINTER(vp),
                                       C.POINTER(vp), vp]
    lib.hdd_multi_info.argtypes = [vp, pi32, pi32]
    lib.hdd_data_scratch_size.argtypes = [vp, i32, C.POINTER(C.c_size_t)]
    lib.hdd_solve_data.argtypes = [vp, i32, vp, vp, vp, vp, vp, i32, vp, vp, vp]
    lib.hdd_profile_begin.argtypes = [vp]
    lib.hdd_profile_end.argtypes = [vp, C.POINTER(KernelStat), i32, C.POINTER(i32)]
    lib.hdd_plan_info.argtypes = [vp, C.POINTER(PlanInfo)]
    lib.hdd_node_info.argtypes = [vp, i32, C.POINTER(NodeInfo)]
    lib.hdd_node_indices.argtypes = [vp, i32, pi32, pi32]
    lib.hdd_status_string.argtypes = [i32]
    lib.hdd_status_string.restype = C.c_char_p
    lib.hdd_last_error.restype = C.c_char_p
    for name in EXPORTED:
        if name not in ("hdd_status_string", "hdd_last_error"):
            getattr(lib, name).restype = i32
    _lib = lib
    return lib


class HDDError(RuntimeError):
    def __init__(self, status: int, where: str):
        lib = load_library()
        msg = lib.hdd_status_string(status).decode()
        detail = lib.hdd_last_error().decode()
        super().__init__(f"{where}: {msg} ({status}) {detail}")
        self.status = status


def _check(status: int, where: str):
    if status != HDD_OK:
        raise HDDError(status, where)


def _ptr(t) -> int:
    return 0 if t is None else int(t.data_ptr())


def _need(t, name: str, dtype: str, shape: tuple, device=None):
    """Raise ValueError unless t is a contiguous tensor of that dtype, exact shape and
    (if given) device: the C ABI takes bare pointers, so a wrong tensor would be read
    or written out of bounds."""
    import torch
    dt = {"f64": torch.float64, "i32": torch.int32}[dtype]
    if t is None or not isinstance(t, torch.Tensor):
        raise ValueError(f"{name} must be a torch tensor")
    if t.dtype != dt or not t.is_contiguous() or tuple(t.shape) != tuple(shape):
        raise ValueError(f"{name} must be a contiguous {dt} tensor of shape {tuple(shape)} "
                         f"(got {t.dtype}, {tuple(t.shape)}, contiguous={t.is_contiguous()})")
    if device is not None and t.device != device:
        raise ValueError(f"{name} must be on {device} (got {t.device})")


def _stream_ptr(stream) -> int:
    """cudaStream_t of a torch stream, an int handle, or torch's current stream (None)."""
    if isinstance(stream, int):
        return stream
    if stream is None:
        import torch
        if not torch.cuda.is_available():
            return 0
        return int(torch.cuda.current_stream().cuda_stream)
    return int(stream.cuda_stream)


class Plan:
    """A device-resident HDD plan for one grid, KL basis and observation set."""

    def __init__(self, N: int, leaf: int, phi: np.ndarray | None, obs: np.ndarray, sigma: float,
                 f: float = 1.0, precision: int = HDD_FP64, ir_max_iter: int = 2, ir_tol: float = 1e-8,
                 fp64_top_levels: int = 0, fuse_height: int = 0, device: int = 0, obs_kind: int = HDD_OBS_VERTEX):
        """obs: vertex ids (obs_kind HDD_OBS_VERTEX) or tree node ids whose mean values are
        observed (HDD_OBS_MEANS; node ids as reported by node() of a plan of the same N, leaf)."""
        self.lib = load_library()
        self.N, self.leaf, self.sigma, self.f = N, leaf, float(sigma), float(f)
        self.obs = np.ascontiguousarray(obs, dtype=np.int32)
        self.n_obs = int(self.obs.size)
        self.device = device
        desc = PlanDesc()
        desc.N, desc.leaf = N, leaf
        if phi is not None:
            self._phi = np.ascontiguousarray(phi, dtype=np.float64)
            desc.n_z = self._phi.shape[1]
            desc.kl_basis = self._phi.ctypes.data_as(C.POINTER(C.c_double))
        else:
            desc.n_z = 1
            desc.kl_basis = None
        self.n_z = desc.n_z
        desc.f = self.f
        desc.n_obs = self.n_obs
        desc.obs_vertex = self.obs.ctypes.data_as(C.POINTER(C.c_int32))
        desc.sigma = self.sigma
        desc.precision, desc.ir_max_iter, desc.ir_tol = precision, ir_max_iter, ir_tol
        desc.fp64_top_levels = fp64_top_levels
        desc.fuse_height = fuse_height
        desc.device = device
        desc.obs_kind = obs_kind
        self.obs_kind = obs_kind
        self.precision = precision
        h = C.c_void_p()
        _check(self.lib.hdd_plan(C.byref(desc), C.byref(h)), "hdd_plan")
        self._h = h
        self._phi = None  # copied by the library

    def close(self):
        if getattr(self, "_h", None):
            self.lib.hdd_plan_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def set_wait_bound(self, polls: int = 1 << 24, stall_node: int = -1, stall_sample: int = -1):
        """hdd_set_wait_bound: polls of each bounded device wait; (stall_node, stall_sample)
        is the test hook that makes one wait run out (-1: off)."""
        _check(self.lib.hdd_set_wait_bound(self._h, polls, stall_node, stall_sample), "hdd_set_wait_bound")

    def set_sweep_fusion(self, max_height: int = 2):
        """hdd_set_sweep_fusion: full sweeps over bottom subtrees of height <= max_height in
        one kernel (0: level by level); info()["sweep_fuse_height"] is the height in use."""
        _check(self.lib.hdd_set_sweep_fusion(self._h, max_height), "hdd_set_sweep_fusion")

    # ---- per-kernel timing ---------------------------------------------
    def profile_begin(self):
        _check(self.lib.hdd_profile_begin(self._h), "hdd_profile_begin")

    def profile_end(self) -> dict:
        """{family: {"launches", "ms", "flops"}} of the kernels launched since profile_begin."""
        arr = (KernelStat * 32)()
        n = C.c_int32()
        _check(self.lib.hdd_profile_end(self._h, arr, 32, C.byref(n)), "hdd_profile_end")
        return {arr[k].name.decode(): {"launches": arr[k].launches, "ms": arr[k].ms, "flops": arr[k].flops}
                for k in range(min(n.value, 32))}

    # ---- queries -------------------------------------------------------
    def info(self) -> dict:
        pi = PlanInfo()
        _check(self.lib.hdd_plan_info(self._h, C.byref(pi)), "hdd_plan_info")
        return {n: getattr(pi, n) for n, _ in PlanInfo._fields_}

    def node(self, k: int) -> dict:
        ni = NodeInfo()
        _check(self.lib.hdd_node_info(self._h, k, C.byref(ni)), "hdd_node_info")
        return {n: getattr(ni, n) for n, _ in NodeInfo._fields_}

    def node_indices(self, k: int):
        d = self.node(k)
        g = np.zeros(d["m"], dtype=np.int32)
        b = np.zeros(d["b"], dtype=np.int32)
        _check(self.lib.hdd_node_indices(self._h, k, g.ctypes.data_as(C.POINTER(C.c_int32)),
                                         b.ctypes.data_as(C.POINTER(C.c_int32))), "hdd_node_indices")
        return g, b

    def workspace_size(self, batch: int) -> int:
        n = C.c_size_t()
        _check(self.lib.hdd_workspace_size(self._h, batch, C.byref(n)), "hdd_workspace_size")
        return int(n.value)

    # ---- device calls (torch tensors on this plan's device) --------------
    def workspace(self, batch: int):
        import torch
        return torch.empty(self.workspace_size(batch), dtype=torch.uint8, device=f"cuda:{self.device}")

    def _dev(self):
        import torch
        return torch.device("cuda", self.device)

    def _check_y(self, y, batch):
        if y is None or y.dim() not in (1, 2):
            raise ValueError("y must be [n_obs] or [batch, n_obs]")
        _need(y, "y", "f64", (self.n_obs,) if y.dim() == 1 else (batch, self.n_obs), self._dev())

    def assemble(self, Z, ws, stream=None):
        batch = Z.shape[0] if Z is not None and Z.dim() == 2 else 0
        _need(Z, "Z", "f64", (batch, self.n_z), self._dev())
        _check(self.lib.hdd_assemble(self._h, _ptr(Z), batch, _ptr(ws), _stream_ptr(stream)), "hdd_assemble")

    def kappa(self, batch: int, ws, out, stream=None):
        """Copy the coefficient field of the last assembly into out (device [batch, n_t] FP64)."""
        _check(self.lib.hdd_kappa(self._h, batch, _ptr(ws), _ptr(out), _stream_ptr(stream)), "hdd_kappa")

    def upsweep(self, batch: int, ws, stream=None):
        _check(self.lib.hdd_upsweep(self._h, batch, _ptr(ws), _stream_ptr(stream)), "hdd_upsweep")

    def point_solve(self, batch: int, ws, u_obs, stream=None):
        _need(u_obs, "u_obs", "f64", (batch, self.n_obs), self._dev())
        _check(self.lib.hdd_point_solve(self._h, batch, _ptr(ws), _ptr(u_obs), _stream_ptr(stream)),
               "hdd_point_solve")

    def solve_loads(self, batch: int, ws, c, u, status=None, stream=None):
        """hdd_solve_loads: c and u device [batch, n_loads, N*N] FP64 (after assemble + upsweep on ws)."""
        import torch
        if c.shape != u.shape or c.dim() != 3 or c.shape[0] != batch or c.shape[2] != self.N * self.N:
            raise ValueError("c and u must both be [batch, n_loads, N*N]")
        if c.dtype != torch.float64 or u.dtype != torch.float64 or not (c.is_contiguous() and u.is_contiguous()):
            raise ValueError("c and u must be contiguous float64 tensors")
        if status is not None and (status.dtype != torch.int32 or status.numel() < batch):
            raise ValueError("status must be an int32 tensor of at least batch entries")
        _check(self.lib.hdd_solve_loads(self._h, batch, _ptr(ws), _ptr(c), int(c.shape[1]), _ptr(u), _ptr(status),
                                        _stream_ptr(stream)), "hdd_solve_loads")

    def solve_data(self, batch: int, ws, u, c=None, f_coarse=None, g=None, status=None, scratch=None, stream=None):
        """hdd_solve_data (after assemble + upsweep on ws): exactly one of c [batch, n_loads, N*N]
        and f_coarse [batch, n_loads, NH*NH] (NH = (N+1)/2), optional g [batch, n_loads, N*N];
        u [batch, n_loads, N*N] out.  scratch: a uint8 device tensor of at least
        data_scratch_size(batch) bytes (allocated here when None)."""
        import torch
        if u.dim() != 3:
            raise ValueError("u must be [batch, n_loads, N*N]")
        nl = int(u.shape[1])
        NN = self.N * self.N
        _need(u, "u", "f64", (batch, nl, NN), self._dev())
        if (c is None) == (f_coarse is None):
            raise ValueError("give exactly one of c and f_coarse")
        if c is not None:
            _need(c, "c", "f64", (batch, nl, NN), self._dev())
        else:
            NH = (self.N + 1) // 2
            _need(f_coarse, "f_coarse", "f64", (batch, nl, NH * NH), self._dev())
        if g is not None:
            _need(g, "g", "f64", (batch, nl, NN), self._dev())
        if status is not None:
            _need(status, "status", "i32", (batch,), self._dev())
        need = self.data_scratch_size(batch)
        if scratch is None:
            scratch = torch.empty(need, dtype=torch.uint8, device=self._dev())
        elif scratch.numel() < need or scratch.device != self._dev():
            raise ValueError(f"scratch must hold {need} bytes on {self._dev()}")
        _check(self.lib.hdd_solve_data(self._h, batch, _ptr(ws), _ptr(scratch), _ptr(c), _ptr(f_coarse), _ptr(g), nl,
                                       _ptr(u), _ptr(status), _stream_ptr(stream)), "hdd_solve_data")

    def data_scratch_size(self, batch: int) -> int:
        n = C.c_size_t()
        _check(self.lib.hdd_data_scratch_size(self._h, batch, C.byref(n)), "hdd_data_scratch_size")
        return int(n.value)

    def subdomain_means(self, u, means, stream=None):
        """hdd_subdomain_means: u device [batch, N*N] (any row stride), means device [batch, n_nodes]."""
        import torch
        if u.dim() != 2 or u.stride(1) != 1 or u.shape[1] != self.N * self.N or u.dtype != torch.float64:
            raise ValueError("u must be float64 [batch, N*N] with unit column stride")
        n_nodes = self.info()["n_nodes"]
        if means.dtype != torch.float64 or not means.is_contiguous() or tuple(means.shape) != (u.shape[0], n_nodes):
            raise ValueError("means must be a contiguous float64 [batch, n_nodes] tensor")
        _check(self.lib.hdd_subdomain_means(self._h, int(u.shape[0]), _ptr(u), int(u.stride(0)), _ptr(means),
                                            _stream_ptr(stream)), "hdd_subdomain_means")

    def mean_functionals(self, batch: int, ws, stream=None):
        """hdd_mean_functionals: (lambda^g of the observed nodes [batch, sum b], mu^f of every
        node [batch, n_nodes]) as the last point_solve on ws left them (mean plans only)."""
        import torch
        nb = sum(self.node(int(k))["b"] for k in self.obs)
        lam = torch.empty(batch, nb, dtype=torch.float64, device=self._dev())
        mu = torch.empty(batch, self.info()["n_nodes"], dtype=torch.float64, device=self._dev())
        _check(self.lib.hdd_mean_functionals(self._h, batch, _ptr(ws), _ptr(lam) if nb else None, _ptr(mu),
                                             _stream_ptr(stream)), "hdd_mean_functionals")
        return lam, mu

    def nodes_at_depth(self, depth: int) -> np.ndarray:
        """Ids of the tree nodes at one depth (the cells of a coarse level), ascending."""
        n = self.info()["n_nodes"]
        return np.array([k for k in range(n) if self.node(k)["depth"] == depth], dtype=np.int32)

    def loglik(self, batch: int, ws, u_obs, y, loglik, status=None, stream=None):
        _need(u_obs, "u_obs", "f64", (batch, self.n_obs), self._dev())
        self._check_y(y, batch)
        _need(loglik, "loglik", "f64", (batch,), self._dev())
        if status is not None:
            _need(status, "status", "i32", (batch,), self._dev())
        per_sample = 1 if y.dim() == 2 else 0
        _check(self.lib.hdd_loglik(self._h, batch, _ptr(ws), _ptr(u_obs), _ptr(y), per_sample, _ptr(loglik),
                                   _ptr(status), _stream_ptr(stream)), "hdd_loglik")

    def evaluate(self, Z, y, ws=None, stream=None):
        """Device tensors in, (loglik [B], u_obs [B, n_obs], status [B]) device tensors out."""
        import torch
        batch = Z.shape[0]
        dev = Z.device
        if ws is None:
            ws = self.workspace(batch)
        u_obs = torch.empty(batch, self.n_obs, dtype=torch.float64, device=dev)
        ll = torch.empty(batch, dtype=torch.float64, device=dev)
        st = torch.empty(batch, dtype=torch.int32, device=dev)
        self.assemble(Z, ws, stream)
        self.upsweep(batch, ws, stream)
        self.point_solve(batch, ws, u_obs, stream)
        self.loglik(batch, ws, u_obs, y, ll, st, stream)
        return ll, u_obs, st

    def evaluate_static(self, Z, y, loglik, u_obs=None, status=None, stream=None):
        """hdd_evaluate_static: same result as evaluate(), workspace in the library's
        static device array (no allocation); device tensors in and out."""
        batch = Z.shape[0] if Z is not None and Z.dim() == 2 else 0
        _need(Z, "Z", "f64", (batch, self.n_z), self._dev())
        self._check_y(y, batch)
        _need(loglik, "loglik", "f64", (batch,), self._dev())
        if u_obs is not None:
            _need(u_obs, "u_obs", "f64", (batch, self.n_obs), self._dev())
        if status is not None:
            _need(status, "status", "i32", (batch,), self._dev())
        per_sample = 1 if y.dim() == 2 else 0
        _check(self.lib.hdd_evaluate_static(self._h, batch, _ptr(Z), _ptr(y), per_sample, _ptr(loglik),
                                            _ptr(u_obs), _ptr(status), _stream_ptr(stream)), "hdd_evaluate_static")

    def evaluate_host_ptrs(self, batch: int, ws, Z_ptr: int, y_ptr: int, y_per_sample: int, ll_ptr: int,
                           uobs_ptr: int, status_ptr: int, stream=None):
        """hdd_evaluate_host on raw host addresses (e.g. pinned torch tensors)."""
        _check(self.lib.hdd_evaluate_host(self._h, batch, _ptr(ws), C.cast(Z_ptr, C.POINTER(C.c_double)),
                                          C.cast(y_ptr, C.POINTER(C.c_double)), y_per_sample,
                                          C.cast(ll_ptr, C.POINTER(C.c_double)),
                                          C.cast(uobs_ptr, C.POINTER(C.c_double)) if uobs_ptr else None,
                                          C.cast(status_ptr, C.POINTER(C.c_int32)) if status_ptr else None,
                                          _stream_ptr(stream)), "hdd_evaluate_host")

    def evaluate_host(self, Z: np.ndarray, y: np.ndarray, ws, stream=None):
        """Host arrays in and out through hdd_evaluate_host (copies inside the call)."""
        Z = np.ascontiguousarray(Z, dtype=np.float64)
        y = np.ascontiguousarray(y, dtype=np.float64)
        batch = Z.shape[0]
        ll = np.empty(batch)
        u_obs = np.empty((batch, self.n_obs))
        st = np.empty(batch, dtype=np.int32)
        dp = C.POINTER(C.c_double)
        _check(self.lib.hdd_evaluate_host(self._h, batch, _ptr(ws), Z.ctypes.data_as(dp), y.ctypes.data_as(dp),
                                          1 if y.ndim == 2 else 0, ll.ctypes.data_as(dp), u_obs.ctypes.data_as(dp),
                                          st.ctypes.data_as(C.POINTER(C.c_int32)), _stream_ptr(stream)),
               "hdd_evaluate_host")
        return ll, u_obs, st


class MultiPlan:
    """Several plans evaluated together (hdd_multi_*): an uneven batch whose "Leaves to Root"
    runs as one launch per tree height and front class over every plan.  Each plan keeps
    its own workspace (allocated here for its batch size)."""

    def __init__(self, plans: list, batches: list):
        import torch
        if len(plans) != len(batches) or not plans:
            raise ValueError("plans and batches must be non-empty lists of the same length")
        self.lib = load_library()
        self.plans = list(plans)
        self.batches = [int(b) for b in batches]
        self.ws = [p.workspace(b) for p, b in zip(self.plans, self.batches)]
        n = len(self.plans)
        hs = (C.c_void_p * n)(*[p._h.value for p in self.plans])
        bs = (C.c_int32 * n)(*self.batches)
        ws = (C.c_void_p * n)(*[w.data_ptr() for w in self.ws])
        h = C.c_void_p()
        _check(self.lib.hdd_multi_create(hs, n, bs, ws, C.byref(h)), "hdd_multi_create")
        self._h = h
        self.outputs = []
        for p, b in zip(self.plans, self.batches):
            dev = p._dev()
            self.outputs.append((torch.empty(b, dtype=torch.float64, device=dev),
                                 torch.empty(b, p.n_obs, dtype=torch.float64, device=dev),
                                 torch.empty(b, dtype=torch.int32, device=dev)))

    def close(self):
        if getattr(self, "_h", None):
            self.lib.hdd_multi_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def info(self) -> dict:
        up, ev = C.c_int32(), C.c_int32()
        _check(self.lib.hdd_multi_info(self._h, C.byref(up), C.byref(ev)), "hdd_multi_info")
        return {"launches_upsweep": up.value, "launches_evaluate": ev.value}

    def upsweep(self, stream=None):
        _check(self.lib.hdd_multi_upsweep(self._h, _stream_ptr(stream)), "hdd_multi_upsweep")

    def evaluate(self, Zs: list, ys: list, stream=None):
        """Device tensors Z_q [batch_q, n_z_q], y_q [n_obs_q] or [batch_q, n_obs_q] in; per plan
        (loglik [batch_q], u_obs [batch_q, n_obs_q], status [batch_q]) out (views of buffers
        that the next call overwrites)."""
        n = len(self.plans)
        if len(Zs) != n or len(ys) != n:
            raise ValueError("one Z and one y per plan")
        for p, b, Z, y in zip(self.plans, self.batches, Zs, ys):
            _need(Z, "Z", "f64", (b, p.n_z), p._dev())
            p._check_y(y, b)
        P = C.c_void_p * n
        ll = P(*[o[0].data_ptr() for o in self.outputs])
        uo = P(*[o[1].data_ptr() for o in self.outputs])
        st = P(*[o[2].data_ptr() for o in self.outputs])
        yps = (C.c_int32 * n)(*[1 if y.dim() == 2 else 0 for y in ys])
        _check(self.lib.hdd_multi_evaluate(self._h, P(*[Z.data_ptr() for Z in Zs]), P(*[y.data_ptr() for y in ys]),
                                           yps, ll, uo, st, _stream_ptr(stream)), "hdd_multi_evaluate")
        return self.outputs

    def capture(self, Zs: list, ys: list):
        """hdd_multi_capture: the evaluation of these Z and y tensors (kept alive by the
        returned graph; write new parameters into them before a launch) as one CUDA graph
        whose results land in self.outputs."""
        n = len(self.plans)
        if len(Zs) != n or len(ys) != n:
            raise ValueError("one Z and one y per plan")
        for p, b, Z, y in zip(self.plans, self.batches, Zs, ys):
            _need(Z, "Z", "f64", (b, p.n_z), p._dev())
            p._check_y(y, b)
        P = C.c_void_p * n
        ll = P(*[o[0].data_ptr() for o in self.outputs])
        uo = P(*[o[1].data_ptr() for o in self.outputs])
        st = P(*[o[2].data_ptr() for o in self.outputs])
        yps = (C.c_int32 * n)(*[1 if y.dim() == 2 else 0 for y in ys])
        h = C.c_void_p()
        _check(self.lib.hdd_multi_capture(self._h, P(*[Z.data_ptr() for Z in Zs]), P(*[y.data_ptr() for y in ys]),
                                          yps, ll, uo, st, C.byref(h)), "hdd_multi_capture")
        return CapturedEvaluation(self, h, list(Zs), list(ys))


class CapturedEvaluation:
    """A captured hdd_multi_evaluate (hdd_multi_capture); launch() replays it on a stream."""

    def __init__(self, multi: "MultiPlan", handle, Zs: list, ys: list):
        self.lib, self.multi, self._h, self.Zs, self.ys = multi.lib, multi, handle, Zs, ys

    def launch(self, stream=None):
        _check(self.lib.hdd_graph_launch(self._h, _stream_ptr(stream)), "hdd_graph_launch")
        return self.multi.outputs

    def close(self):
        if getattr(self, "_h", None):
            self.lib.hdd_graph_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
