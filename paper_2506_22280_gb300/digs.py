"""Thin Python binding of libdigs (include/digs.h): argument marshalling only.

Every step of the hot path runs in the CUDA kernels of ``libdigs.so``; this module turns torch CUDA
tensors into device pointers, scan geometry dicts into ``DigsView`` structs and forwards the call on
torch's current stream.  There is no CPU fallback: if the library is missing, every call raises.
"""
from __future__ import annotations

import ctypes as C
import math
import os
from typing import Dict, List, Optional, Sequence, Tuple

import torch

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libdigs.so")

DIGS_MAX_R = 4
DIGS_MAX_VIEWS = 128
DIGS_MAX_SCANS = 8
DIGS_FLAG_REUSE_BINNING = 1
DIGS_FLAG_EWA = 4
STATUS = {0: "ok", 1: "invalid argument", 2: "CUDA error", 3: "workspace too small for the pairs",
          4: "device-side wait timed out", 5: "non-finite input"}


class DigsError(RuntimeError):
    def __init__(self, code: int, where: str):
        super().__init__(f"{where}: {STATUS.get(code, code)} (status {code})")
        self.code = code


class DigsGaussians(C.Structure):
    _fields_ = [("n", C.c_int), ("mu0", C.c_void_p), ("scale", C.c_void_p), ("quat", C.c_void_p), ("rho", C.c_void_p)]


class DigsLattice(C.Structure):
    _fields_ = [("nx", C.c_int), ("ny", C.c_int), ("nz", C.c_int), ("R", C.c_int),
                ("origin", C.c_float * 3), ("spacing", C.c_float * 3)]


class DigsView(C.Structure):
    _fields_ = [("src", C.c_double * 3), ("det_c", C.c_double * 3), ("e_u", C.c_double * 3), ("e_v", C.c_double * 3),
                ("du", C.c_double), ("dv", C.c_double), ("off_u", C.c_double), ("off_v", C.c_double),
                ("nu", C.c_int), ("nv", C.c_int), ("parallel", C.c_int), ("scan", C.c_int)]


class DigsOpts(C.Structure):
    _fields_ = [("cutoff", C.c_float), ("tile", C.c_int), ("flags", C.c_int), ("bwd_lanes", C.c_int)]


class DigsAdamConfig(C.Structure):
    _fields_ = [("lr0", C.c_float * 6), ("lr1", C.c_float * 6), ("beta1", C.c_float), ("beta2", C.c_float),
                ("eps", C.c_float), ("total_iters", C.c_int)]


class DigsState(C.Structure):
    _fields_ = [("n", C.c_int), ("mu0", C.c_void_p), ("scale", C.c_void_p), ("quat", C.c_void_p), ("rho", C.c_void_p),
                ("phi", C.c_void_p), ("w", C.c_void_p), ("n_w", C.c_int), ("m", C.c_void_p), ("v", C.c_void_p),
                ("grad", C.c_void_p), ("iter", C.c_int), ("lat", DigsLattice), ("adam", DigsAdamConfig),
                ("n_scans", C.c_int), ("scan_off", C.c_int * (DIGS_MAX_SCANS + 1)), ("iter_dev", C.c_void_p),
                ("w_ctrl", C.c_void_p), ("n_ctrl", C.c_int), ("t_step", C.c_float), ("dens_grad", C.c_void_p)]


class DigsDensifyOpts(C.Structure):
    _fields_ = [("tau", C.c_float), ("n_projections", C.c_int), ("s_split", C.c_float), ("rho_min", C.c_float)]


_lib = None


def lib() -> C.CDLL:
    """Load libdigs.so (built in-tree by ``paper_2506_22280_gb300.build``); raise if it is missing."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(LIB_PATH):
        raise RuntimeError(f"{LIB_PATH} is not built; run `python -c 'import __graft_entry__ as g; g.build()'`")
    L = C.CDLL(LIB_PATH)
    P, I, S, LL = C.c_void_p, C.c_int, C.c_size_t, C.c_longlong
    sig = {
        "digs_workspace_size": (S, [I, I, I, I, I, LL, P]),
        "digs_ffd_eval": (I, [P, P, P, I, P, P, P]),
        "digs_count_pairs": (I, [P, P, P, P, P, I, P, P, S, C.POINTER(LL), P]),
        "digs_project_fwd": (I, [P, P, P, P, P, I, P, P, P, S, P]),
        "digs_project_bwd": (I, [P, P, P, P, P, I, P, P, P, P, P, P, P, P, P, S, P]),
        "digs_project_loss": (I, [P, P, P, P, P, I, P, P, P, P, P, S, P]),
        "digs_state_moments": (S, [I, P, I, I]),
        "digs_state_workspace_size": (S, [P, I, I, I, LL, P]),
        "digs_state_size": (S, [P]),
        "digs_step": (I, [P, P, P, P, I, P, P, P, S, P]),
        "digs_sync_status": (I, [P, P]),
        "digs_status_string": (C.c_char_p, [I]),
        "digs_stage_times": (I, [P]),
        "digs_kernel_launches": (LL, []),
        "digs_pair_stats": (I, [P, P, P]),
        "digs_voxelize": (I, [P, P, P, P, P, P, P, P]),
        "digs_dvf": (I, [P, P, P, P, P, P]),
        "digs_cnn_params": (S, [I]),
        "digs_cnn_workspace_size": (S, [I, I]),
        "digs_cnn_init": (I, [P, I, C.c_ulonglong, P]),
        "digs_cnn_prepare_input": (I, [P, I, I, I, C.c_float, P, P]),
        "digs_cnn_forward": (I, [P, I, P, P, I, P, I, P, S, P]),
        "digs_cnn_backward": (I, [P, I, I, P, P, I, P, S, P]),
        "digs_cnn_train_step": (I, [P, P, P, P, I, C.c_float, I, P, P, P, I, P, I, P, S, P]),
        "digs_cnn_infer_bf16": (I, [P, I, P, P, I, P, P, S, P]),
        "digs_gemm_bf16": (I, [I, I, I, I, I, P, I, P, I, P, I, P, I, I, P, P, P]),
        "digs_densify_workspace_size": (S, [I]),
        "digs_densify_plan": (I, [I, P, P, P, P, P, P, P, S, P]),
        "digs_densify_apply": (I, [P, P, P, P, I, P, P, P, P, P, P, P]),
        "digs_gather_rows": (I, [P, P, I, I, P, P, P]),
        "digs_project_fwd_static": (I, [P, P, P, P, P, I, P, P, P]),
        "digs_set_wait_limit": (I, [LL]),
        "digs_pipe_bench": (I, [I, I, P, C.POINTER(LL), P]),
    }
    for name, (res, args) in sig.items():
        f = getattr(L, name)
        f.restype = res
        f.argtypes = args
    _lib = L
    return L


def exported_symbols() -> List[str]:
    return ["digs_workspace_size", "digs_ffd_eval", "digs_count_pairs", "digs_project_fwd", "digs_project_bwd",
            "digs_project_loss",
            "digs_state_moments", "digs_state_workspace_size", "digs_state_size", "digs_step", "digs_sync_status", "digs_status_string", "digs_stage_times",
            "digs_kernel_launches", "digs_pair_stats", "digs_voxelize", "digs_dvf", "digs_cnn_params", "digs_cnn_workspace_size", "digs_cnn_init",
            "digs_cnn_prepare_input", "digs_cnn_forward", "digs_cnn_backward", "digs_cnn_train_step",
            "digs_cnn_infer_bf16", "digs_gemm_bf16", "digs_densify_workspace_size", "digs_densify_plan",
            "digs_densify_apply", "digs_gather_rows", "digs_project_fwd_static", "digs_set_wait_limit",
            "digs_pipe_bench"]


DIGS_FLAG_TIME_STAGES = 2
STAGES = ["setup", "bin", "order", "raster_fwd", "loss", "raster_bwd", "chain_bwd", "adam"]


def stage_times() -> Dict[str, float]:
    """Milliseconds per stage of the most recent call made with time_stages=True (synchronises)."""
    arr = (C.c_float * len(STAGES))()
    _check(lib().digs_stage_times(arr), "digs_stage_times")
    return {k: float(arr[i]) for i, k in enumerate(STAGES)}


PIPES = ("ffma", "ffma2", "ex2", "rsqrt")


def pipe_rate(kind: str, iters: int = 4096, reps: int = 3) -> float:
    """FP32 results per second of one arithmetic pipe (digs_pipe_bench): the best of `reps` launches,
    each timed with CUDA events on the current stream after one untimed launch."""
    k = PIPES.index(kind)
    sink = torch.zeros(1, device="cuda")
    ops = C.c_longlong(0)
    best = 0.0
    for r in range(reps + 1):
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        _check(lib().digs_pipe_bench(k, int(iters), _ptr(sink), C.byref(ops), _stream()), "digs_pipe_bench")
        e1.record()
        e1.synchronize()
        if r > 0:
            best = max(best, ops.value / (e0.elapsed_time(e1) / 1e3))
    return best


def set_wait_limit(tests: int) -> None:
    """Tests a tensor-core GEMM K-loop wait makes before it gives up (< 0: the default)."""
    _check(lib().digs_set_wait_limit(int(tests)), "digs_set_wait_limit")


def kernel_launches() -> int:
    return int(lib().digs_kernel_launches())


def pair_stats(ws: "Workspace") -> Dict[str, int]:
    """Pairs binned into tiles, pixel-box pairs evaluated and pairs within the cutoff in the last forward."""
    out = (C.c_longlong * 3)()
    _check(lib().digs_pair_stats(ws.ptr, out, _stream()), "digs_pair_stats")
    return dict(tile_pairs=int(out[0]), box_pairs=int(out[1]), cutoff_pairs=int(out[2]))


# ----------------------------------------------------------------------------- marshalling helpers
def _ptr(t: Optional[torch.Tensor]):
    if t is None:
        return None
    if not t.is_cuda:
        raise ValueError("libdigs takes CUDA tensors")
    if not t.is_contiguous():
        raise ValueError("libdigs takes contiguous tensors")
    return C.c_void_p(t.data_ptr())


def _f32(t: torch.Tensor, name: str) -> torch.Tensor:
    if t.dtype != torch.float32:
        raise TypeError(f"{name} must be float32, got {t.dtype}")
    return t


def _stream():
    return C.c_void_p(torch.cuda.current_stream().cuda_stream)


def _check(code: int, where: str):
    if code != 0:
        raise DigsError(code, where)


def lattice_struct(lat: Dict) -> DigsLattice:
    s = DigsLattice()
    s.nx, s.ny, s.nz, s.R = int(lat["nx"]), int(lat["ny"]), int(lat["nz"]), int(lat["R"])
    for a in range(3):
        s.origin[a] = float(lat["origin"][a])
        s.spacing[a] = float(lat["spacing"][a])
    return s


def views_array(views: Sequence[Dict]):
    arr = (DigsView * max(len(views), 1))()
    for i, v in enumerate(views):
        d = arr[i]
        for key in ("src", "det_c", "e_u", "e_v"):
            vec = getattr(d, key)
            for a in range(3):
                vec[a] = float(v[key][a])
        d.du, d.dv = float(v["du"]), float(v["dv"])
        d.off_u, d.off_v = float(v.get("off_u", 0.0)), float(v.get("off_v", 0.0))
        d.nu, d.nv = int(v["nu"]), int(v["nv"])
        d.parallel = 1 if v.get("parallel", False) else 0
        d.scan = int(v.get("scan", 0))
    return arr


def opts_struct(cutoff: float = 3.5, tile: int = 16, flags: int = 0, bwd_lanes: int = 16) -> DigsOpts:
    return DigsOpts(float(cutoff), int(tile), int(flags), int(bwd_lanes))


def gauss_struct(mu0, scale, quat, rho) -> DigsGaussians:
    return DigsGaussians(int(mu0.shape[0]), _ptr(_f32(mu0, "mu0")), _ptr(_f32(scale, "scale")),
                         _ptr(_f32(quat, "quat")), _ptr(_f32(rho, "rho")))


# ----------------------------------------------------------------------------- entry points
def workspace_size(n: int, P: int, nu: int, nv: int, R: int, max_pairs: int, cutoff=3.5, tile=16) -> int:
    o = opts_struct(cutoff, tile)
    return int(lib().digs_workspace_size(n, P, nu, nv, R, int(max_pairs), C.byref(o)))


def ffd_eval(phi: torch.Tensor, lattice: Dict, x: torch.Tensor):
    """u_r(x) [n][R][3] and grad u_r(x) [n][R][3][3] (Eq. 10-11), one CUDA thread per point."""
    R = int(lattice["R"])
    n = int(x.shape[0])
    U = torch.empty(n, R, 3, device=x.device, dtype=torch.float32)
    dU = torch.empty(n, R, 3, 3, device=x.device, dtype=torch.float32)
    lat = lattice_struct(lattice)
    _check(lib().digs_ffd_eval(C.byref(lat), _ptr(_f32(phi, "phi")), _ptr(_f32(x, "x")), n, _ptr(U), _ptr(dU),
                               _stream()), "digs_ffd_eval")
    return U, dU


class Workspace:
    """Caller-owned scratch memory for libdigs calls (a zero-initialised torch uint8 buffer)."""

    def __init__(self, device="cuda"):
        self.device = torch.device(device)
        self.buf: Optional[torch.Tensor] = None

    def ensure(self, nbytes: int) -> "Workspace":
        nbytes = int(nbytes)
        if self.buf is None or self.buf.numel() < nbytes:
            self.buf = torch.zeros(nbytes + 256, dtype=torch.uint8, device=self.device)
        return self

    @property
    def ptr(self):
        base = self.buf.data_ptr()
        return C.c_void_p((base + 255) & ~255)

    @property
    def nbytes(self) -> int:
        base = self.buf.data_ptr()
        return int(self.buf.numel() - (((base + 255) & ~255) - base))


def sync_status(ws: Workspace) -> int:
    return int(lib().digs_sync_status(ws.ptr, _stream()))


class Projector:
    """Forward / backward projection of one Gaussian set through the C-ABI, keeping a workspace sized
    by the pair count of the inputs it last saw (recounted when a call reports overflow)."""

    def __init__(self, lattice: Dict, views: Sequence[Dict], cutoff: float = 3.5, tile: int = 16,
                 headroom: float = 1.25, device="cuda", bwd_lanes: int = 16, ewa: bool = False):
        if len(views) > DIGS_MAX_VIEWS:
            raise ValueError(f"at most {DIGS_MAX_VIEWS} views per call")
        self.lattice = dict(lattice)
        self.lat = lattice_struct(lattice)
        self.views = list(views)
        self.varr = views_array(self.views)
        self.P = len(self.views)
        self.nu = int(self.views[0]["nu"]) if self.views else 1
        self.nv = int(self.views[0]["nv"]) if self.views else 1
        self.model = DIGS_FLAG_EWA if ewa else 0  # the paper's 2D-Gaussian model instead of the exact integral
        self.opts = opts_struct(cutoff, tile, self.model, bwd_lanes)
        self.cutoff, self.tile, self.headroom, self.bwd_lanes = cutoff, tile, headroom, bwd_lanes
        self.ws = Workspace(device)
        self.cap = -1

    def set_views(self, views: Sequence[Dict]) -> None:
        """Project along other views of the same count and detector (the workspace is kept; call
        reserve(force=True) if the pair count may have grown)."""
        if len(views) != self.P:
            raise ValueError("set_views keeps the number of views")
        self.views = list(views)
        self.varr = views_array(self.views)

    def _size(self, n, cap):
        return workspace_size(n, self.P, self.nu, self.nv, int(self.lattice["R"]), cap, self.cutoff, self.tile)

    def count_pairs(self, mu0, scale, quat, rho, phi, w) -> int:
        n = int(mu0.shape[0])
        self.ws.ensure(self._size(n, 0))
        g = gauss_struct(mu0, scale, quat, rho)
        out = C.c_longlong(0)
        _check(lib().digs_count_pairs(C.byref(g), C.byref(self.lat), _ptr(_f32(phi, "phi")), _ptr(_f32(w, "w")),
                                      self.varr, self.P, C.byref(self.opts), self.ws.ptr, self.ws.nbytes,
                                      C.byref(out), _stream()), "digs_count_pairs")
        return int(out.value)

    def reserve(self, mu0, scale, quat, rho, phi, w, force: bool = False) -> int:
        n = int(mu0.shape[0])
        if force or self.cap < 0:
            cnt = self.count_pairs(mu0, scale, quat, rho, phi, w)
            self.cap = int(math.ceil(cnt * self.headroom)) + 1024
            self.ws.ensure(self._size(n, self.cap))
        return self.cap

    def forward(self, mu0, scale, quat, rho, phi, w, out: Optional[torch.Tensor] = None) -> torch.Tensor:
        self.reserve(mu0, scale, quat, rho, phi, w)
        if out is None:
            out = torch.empty(self.P, self.nv, self.nu, device=mu0.device, dtype=torch.float32)
        g = gauss_struct(mu0, scale, quat, rho)
        _check(lib().digs_project_fwd(C.byref(g), C.byref(self.lat), _ptr(_f32(phi, "phi")), _ptr(_f32(w, "w")),
                                      self.varr, self.P, C.byref(self.opts), _ptr(out), self.ws.ptr, self.ws.nbytes,
                                      _stream()), "digs_project_fwd")
        return out

    def loss(self, mu0, scale, quat, rho, phi, w, meas: torch.Tensor, out: Optional[torch.Tensor] = None,
             proj: Optional[torch.Tensor] = None) -> torch.Tensor:
        """Mean over the views' pixels of (I - meas)^2 (device tensor [1]), the residuals squared and
        summed in the raster kernel (digs_project_loss); proj, if given, receives I."""
        self.reserve(mu0, scale, quat, rho, phi, w)
        if out is None:
            out = torch.empty(1, device=mu0.device, dtype=torch.float32)
        g = gauss_struct(mu0, scale, quat, rho)
        _check(lib().digs_project_loss(C.byref(g), C.byref(self.lat), _ptr(_f32(phi, "phi")), _ptr(_f32(w, "w")),
                                       self.varr, self.P, C.byref(self.opts), _ptr(_f32(meas.contiguous(), "meas")),
                                       _ptr(proj), _ptr(out), self.ws.ptr, self.ws.nbytes, _stream()),
               "digs_project_loss")
        return out

    def backward(self, mu0, scale, quat, rho, phi, w, grad_proj, reuse: bool = False):
        self.reserve(mu0, scale, quat, rho, phi, w)
        n = int(mu0.shape[0])
        dev = mu0.device
        g_mu0 = torch.empty(n, 3, device=dev)
        g_scale = torch.empty(n, 3, device=dev)
        g_quat = torch.empty(n, 4, device=dev)
        g_rho = torch.empty(n, device=dev)
        g_phi = torch.empty_like(phi)
        g_w = torch.empty(self.P, int(self.lattice["R"]), device=dev)
        g = gauss_struct(mu0, scale, quat, rho)
        o = opts_struct(self.cutoff, self.tile, self.model | (DIGS_FLAG_REUSE_BINNING if reuse else 0),
                        self.bwd_lanes)
        _check(lib().digs_project_bwd(C.byref(g), C.byref(self.lat), _ptr(_f32(phi, "phi")), _ptr(_f32(w, "w")),
                                      self.varr, self.P, C.byref(o), _ptr(_f32(grad_proj.contiguous(), "grad_proj")),
                                      _ptr(g_mu0), _ptr(g_scale), _ptr(g_quat), _ptr(g_rho), _ptr(g_phi), _ptr(g_w),
                                      self.ws.ptr, self.ws.nbytes, _stream()), "digs_project_bwd")
        return dict(mu0=g_mu0, scale=g_scale, quat=g_quat, rho=g_rho, phi=g_phi, w=g_w)

    def status(self) -> int:
        return sync_status(self.ws)


class DigsRender(torch.autograd.Function):
    """Differentiable projection: ``DigsRender.apply(projector, mu0, scale, quat, rho, phi, w)`` returns
    the projections [P][nv][nu]; its backward runs the hand-written CUDA backward (tile lists are rebuilt
    in the backward rather than stored)."""

    @staticmethod
    def forward(ctx, projector: Projector, mu0, scale, quat, rho, phi, w):
        ctx.projector = projector
        ctx.save_for_backward(mu0, scale, quat, rho, phi, w)
        return projector.forward(mu0, scale, quat, rho, phi, w)

    @staticmethod
    def backward(ctx, grad_out):
        mu0, scale, quat, rho, phi, w = ctx.saved_tensors
        g = ctx.projector.backward(mu0, scale, quat, rho, phi, w, grad_out.contiguous())
        return None, g["mu0"], g["scale"], g["quat"], g["rho"], g["phi"], g["w"]


def adam_config(lr0: Sequence[float], lr1: Sequence[float], total_iters: int, beta1=0.9, beta2=0.999,
                eps=1e-15) -> DigsAdamConfig:
    c = DigsAdamConfig()
    for k in range(6):
        c.lr0[k] = float(lr0[k])
        c.lr1[k] = float(lr1[k])
    c.beta1, c.beta2, c.eps, c.total_iters = float(beta1), float(beta2), float(eps), int(total_iters)
    return c


class Reconstruction:
    """Parameters, Adam moments and gradient scratch of one reconstruction in device memory, stepped by
    ``digs_step`` (render a batch, L2 loss, backward, fused Adam).

    Several independent scans may share the state (``scan_sizes`` = their Gaussian counts, stacked in that
    order in mu0 / scale / quat / rho; ``phi`` is then [S][R][nz][ny][nx][3] and ``w`` holds the weight rows
    of every scan's projections); each view of a batch names its scan in ``view["scan"]``, and one step
    renders the projections of all scans with one launch per stage."""

    def __init__(self, mu0, scale, quat, rho, phi, w, lattice: Dict, adam: DigsAdamConfig, cutoff=3.5, tile=16,
                 headroom=1.3, device="cuda", scan_sizes: Optional[Sequence[int]] = None, bwd_lanes: int = 16,
                 w_ctrl=None, t_step: float = 4.0):
        dev = torch.device(device)
        f = lambda a: torch.as_tensor(a, dtype=torch.float32, device=dev).contiguous().clone()
        self.mu0, self.scale, self.quat, self.rho = f(mu0), f(scale), f(quat), f(rho)
        self.phi, self.w = f(phi), f(w)
        self.lattice = dict(lattice)
        self.lat = lattice_struct(lattice)
        n = int(self.mu0.shape[0])
        sizes = [n] if scan_sizes is None else [int(k) for k in scan_sizes]
        if sum(sizes) != n or not 1 <= len(sizes) <= DIGS_MAX_SCANS:
            raise ValueError("scan_sizes must add up to the number of Gaussians (at most %d scans)" % DIGS_MAX_SCANS)
        self.scan_off = [0]
        for k in sizes:
            self.scan_off.append(self.scan_off[-1] + k)
        self.S = len(sizes)
        if self.S > 1:
            self.phi = self.phi.reshape(self.S, -1)
        self.n_w = int(self.w.shape[0])
        self.w_ctrl = None if w_ctrl is None else f(w_ctrl)
        self.t_step = float(t_step)
        self.state = DigsState()
        self.state.n = n
        self.state.mu0, self.state.scale = self.mu0.data_ptr(), self.scale.data_ptr()
        self.state.quat, self.state.rho = self.quat.data_ptr(), self.rho.data_ptr()
        self.state.phi, self.state.w, self.state.n_w = self.phi.data_ptr(), self.w.data_ptr(), self.n_w
        self.state.iter = 0
        self.state.lat = self.lat
        self.state.adam = adam
        self.state.n_scans = self.S if self.S > 1 else 0
        for k, o in enumerate(self.scan_off):
            self.state.scan_off[k] = o
        if self.w_ctrl is not None:  # weights from temporal B-spline control points (one scan)
            self.state.w_ctrl, self.state.n_ctrl = self.w_ctrl.data_ptr(), int(self.w_ctrl.shape[0])
            self.state.t_step = self.t_step
        nm = int(lib().digs_state_size(C.byref(self.state)))
        self.m = torch.zeros(nm, device=dev)
        self.v = torch.zeros(nm, device=dev)
        self.grad = torch.zeros(nm, device=dev)
        self.state.m, self.state.v, self.state.grad = self.m.data_ptr(), self.v.data_ptr(), self.grad.data_ptr()
        self.cutoff, self.tile, self.headroom, self.bwd_lanes = cutoff, tile, headroom, bwd_lanes
        self.ws = Workspace(dev)
        self.cap = {}
        self.loss = torch.zeros(1, device=dev)
        self.dens_grad = None
        self.dens_projections = 0

    def scan_params(self, s: int) -> Dict[str, torch.Tensor]:
        """Views of scan s's Gaussians and control points inside the state."""
        a, b = self.scan_off[s], self.scan_off[s + 1]
        phi = self.phi[s] if self.S > 1 else self.phi
        return dict(mu0=self.mu0[a:b], scale=self.scale[a:b], quat=self.quat[a:b], rho=self.rho[a:b],
                    phi=phi.reshape(-1))

    def count_pairs(self, views, proj_ids) -> int:
        """(tile, Gaussian) pairs of one batch with the current parameters (synchronises)."""
        total = 0
        for s in range(self.S):
            sel = [k for k, v in enumerate(views) if int(v.get("scan", 0)) == s]
            if not sel:
                continue
            pj = Projector(self.lattice, [views[k] for k in sel], self.cutoff, self.tile, self.headroom,
                           self.mu0.device)
            p = self.scan_params(s)
            w_rows = self.w[torch.as_tensor([proj_ids[k] for k in sel], device=self.w.device)].contiguous()
            total += pj.count_pairs(p["mu0"], p["scale"], p["quat"], p["rho"], p["phi"], w_rows)
        return total

    def workspace_bytes(self, B: int, nu: int, nv: int, max_pairs: int) -> int:
        o = opts_struct(self.cutoff, self.tile)
        return int(lib().digs_state_workspace_size(C.byref(self.state), B, nu, nv, int(max_pairs), C.byref(o)))

    def _reserve(self, views, B, proj_ids):
        key = B
        if key in self.cap:
            return
        cap = int(math.ceil(self.count_pairs(views, proj_ids) * self.headroom)) + 4096
        nu, nv = int(views[0]["nu"]), int(views[0]["nv"])
        self.ws.ensure(self.workspace_bytes(B, nu, nv, cap))
        self.cap[key] = cap

    def step(self, meas: torch.Tensor, proj_ids: Sequence[int], views: Sequence[Dict], time_stages: bool = False,
             varr=None) -> torch.Tensor:
        """One iteration over the batch; returns the (device) loss tensor of this step.  ``varr`` may hold
        the pre-marshalled views of the batch."""
        B = len(proj_ids)
        self._reserve(views, B, proj_ids)
        ids = (C.c_int * B)(*[int(i) for i in proj_ids])
        if varr is None:
            varr = views_array(views)
        o = opts_struct(self.cutoff, self.tile, DIGS_FLAG_TIME_STAGES if time_stages else 0, self.bwd_lanes)
        _check(lib().digs_step(C.byref(self.state), _ptr(_f32(meas, "meas")), ids, varr, B, C.byref(o),
                               _ptr(self.loss), self.ws.ptr, self.ws.nbytes, _stream()), "digs_step")
        if self.dens_grad is not None:
            self.dens_projections += B
        return self.loss

    # ---- adaptive density control ----------------------------------------------------------------
    def enable_density_stats(self) -> None:
        """Let every step add the density-control statistic (sum over its projections of |dL/dmu'|) into
        ``dens_grad`` (one scan only)."""
        if self.S != 1:
            raise ValueError("density control is for one-scan states")
        self.dens_grad = torch.zeros(int(self.mu0.shape[0]), device=self.mu0.device)
        self.dens_projections = 0
        self.state.dens_grad = self.dens_grad.data_ptr()

    def densify(self, tau: float = 5e-8, s_split: float = 4.0, rho_min: float = 1e-5,
                generator: Optional[torch.Generator] = None) -> Dict[str, int]:
        """Prune, clone and split Gaussians by the statistic gathered since the last call
        (include/digs.h, "Adaptive density control"); the Adam moments of kept Gaussians carry over, new
        ones start at zero, the statistic restarts.  Captured graphs of earlier steps no longer apply."""
        if self.dens_grad is None or self.dens_projections < 1:
            raise ValueError("enable_density_stats() and at least one step first")
        n = int(self.mu0.shape[0])
        action, dst = densify_plan(self.dens_grad, self.scale, self.rho, tau, self.dens_projections, s_split, rho_min)
        n_out = int(dst[n].item())
        z = torch.randn(n, 2, 3, device=self.mu0.device, generator=generator)
        out = densify_apply(self.mu0, self.scale, self.quat, self.rho, action, dst, z, n_out)
        src, new = out["src"], out["new"]
        groups = []
        off = 0
        for d in (3, 3, 4, 1):  # mu0, log-scale, quat, density moments, per Gaussian
            groups.append((off, d))
            off += d * n
        m_new, v_new = [], []
        for o, d in groups:
            m_new.append(gather_rows(src, new, self.m[o:o + d * n].view(n, d)).reshape(-1))
            v_new.append(gather_rows(src, new, self.v[o:o + d * n].view(n, d)).reshape(-1))
        self.m = torch.cat(m_new + [self.m[off:]])
        self.v = torch.cat(v_new + [self.v[off:]])
        self.grad = torch.zeros_like(self.m)
        self.mu0, self.scale, self.quat, self.rho = out["mu0"], out["scale"], out["quat"], out["rho"]
        st = self.state
        st.n = n_out
        st.mu0, st.scale, st.quat, st.rho = (self.mu0.data_ptr(), self.scale.data_ptr(), self.quat.data_ptr(),
                                             self.rho.data_ptr())
        st.m, st.v, st.grad = self.m.data_ptr(), self.v.data_ptr(), self.grad.data_ptr()
        self.scan_off = [0, n_out]
        st.scan_off[1] = n_out
        self.dens_grad = torch.zeros(n_out, device=self.mu0.device)
        st.dens_grad = self.dens_grad.data_ptr()
        self.dens_projections = 0
        self.cap = {}
        a = action.cpu()
        return dict(n_before=n, n_after=n_out, pruned=int((a == -1).sum()), cloned=int((a == 1).sum()),
                    split=int((a == 2).sum()))

    def clone(self) -> "Reconstruction":
        """An independent copy of the state (parameters, Adam moments, step count)."""
        sizes = [self.scan_off[k + 1] - self.scan_off[k] for k in range(self.S)]
        r = Reconstruction(self.mu0, self.scale, self.quat, self.rho, self.phi, self.w, self.lattice, self.state.adam,
                           self.cutoff, self.tile, self.headroom, self.mu0.device, sizes if self.S > 1 else None,
                           self.bwd_lanes, self.w_ctrl, self.t_step)
        r.m.copy_(self.m)
        r.v.copy_(self.v)
        r.state.iter = self.iter
        return r

    # ---- graph-captured iterations -------------------------------------------------------------
    def use_device_counter(self) -> None:
        """Keep the step count on the device (the learning-rate schedule and Adam's bias correction then
        come from it), so that a captured step can be replayed."""
        if getattr(self, "iter_dev", None) is None:
            self.iter_dev = torch.full((1,), int(self.state.iter), dtype=torch.int32, device=self.mu0.device)
            self.state.iter_dev = self.iter_dev.data_ptr()

    def capture(self, batches: Sequence[Tuple[torch.Tensor, Sequence[int], Sequence[Dict]]]) -> List["torch.cuda.CUDAGraph"]:
        """One CUDA graph per (measured projections, projection ids, views) batch, each holding a whole
        step (set-up, binning, both rasters, chain, Adam); ``graph.replay()`` runs the step again with the
        current parameters.  The measured tensors are captured by address and kept alive here.  Run at
        least one eager step first (it sizes the workspace and initialises the kernels)."""
        self.use_device_counter()
        for M, ids, views in batches:
            self._reserve(views, len(ids), ids)
        torch.cuda.synchronize()
        graphs = []
        keep = []
        for M, ids, views in batches:
            M = _f32(M, "meas")
            varr = views_array(views)
            g = torch.cuda.CUDAGraph()
            with torch.cuda.graph(g):
                self.step(M, ids, views, varr=varr)
            graphs.append(g)
            keep.append((M, varr))
        self._graph_inputs = getattr(self, "_graph_inputs", []) + keep
        return graphs

    @property
    def iter(self) -> int:
        if getattr(self, "iter_dev", None) is not None:
            return int(self.iter_dev.item())
        return int(self.state.iter)

    def status(self) -> int:
        return sync_status(self.ws)


def gemm_bf16(a: torch.Tensor, b: torch.Tensor, trans_a: bool = False, trans_b: bool = False,
              bias: Optional[torch.Tensor] = None, relu: bool = False, splits: int = 1) -> Tuple[torch.Tensor, torch.Tensor]:
    """C = op(a) op(b) (+ bias, ReLU) on the tensor cores: BF16 operands rounded from a, b (FP32), FP32
    accumulation (include/digs.h, digs_gemm_bf16).  op(a) = a.T if trans_a; op(b) = b.T if trans_b.
    Returns (C [M][N] float32, status [1] int32: nonzero if a bounded wait in the kernel gave up)."""
    a, b = _f32(a, "a").contiguous(), _f32(b, "b").contiguous()
    M, K = (a.shape[1], a.shape[0]) if trans_a else (a.shape[0], a.shape[1])
    Kb, N = (b.shape[1], b.shape[0]) if trans_b else (b.shape[0], b.shape[1])
    if K != Kb:
        raise ValueError(f"inner dimensions differ: {K} vs {Kb}")
    out = torch.empty(M, N, device=a.device, dtype=torch.float32)
    part = torch.empty(splits, M, N, device=a.device, dtype=torch.float32) if splits > 1 else None
    status = torch.zeros(1, device=a.device, dtype=torch.int32)
    _check(lib().digs_gemm_bf16(int(trans_a), int(trans_b), M, N, K, _ptr(a), int(a.shape[1]), _ptr(b),
                                int(b.shape[1]), _ptr(bias), int(relu), _ptr(out), N, int(splits), _ptr(part),
                                _ptr(status), _stream()), "digs_gemm_bf16")
    return out, status


def densify_plan(grad_sum: torch.Tensor, scale: torch.Tensor, rho: torch.Tensor, tau: float, n_projections: int,
                 s_split: float, rho_min: float) -> Tuple[torch.Tensor, torch.Tensor]:
    """Density-control plan (include/digs.h, digs_densify_plan): action [n] (-1 prune, 0 keep, 1 clone,
    2 split) and dst [n + 1] (first output row of each Gaussian; dst[n] = output rows), int32 on the
    device."""
    n = int(scale.shape[0])
    dev = scale.device
    action = torch.empty(n, dtype=torch.int32, device=dev)
    dst = torch.empty(n + 1, dtype=torch.int32, device=dev)
    ws = torch.empty(int(lib().digs_densify_workspace_size(n)), dtype=torch.uint8, device=dev)
    o = DigsDensifyOpts(float(tau), int(n_projections), float(s_split), float(rho_min))
    _check(lib().digs_densify_plan(n, _ptr(_f32(grad_sum, "grad_sum")), _ptr(_f32(scale, "scale")),
                                   _ptr(_f32(rho, "rho")), C.byref(o), _ptr(action), _ptr(dst), _ptr(ws),
                                   int(ws.numel()), _stream()), "digs_densify_plan")
    return action, dst


def densify_apply(mu0, scale, quat, rho, action, dst, z, n_out: int) -> Dict[str, torch.Tensor]:
    """The densified cloud of a plan (digs_densify_apply); z: [n][2][3] standard normal draws."""
    dev = mu0.device
    out = dict(mu0=torch.empty(n_out, 3, device=dev), scale=torch.empty(n_out, 3, device=dev),
               quat=torch.empty(n_out, 4, device=dev), rho=torch.empty(n_out, device=dev),
               src=torch.empty(n_out, dtype=torch.int32, device=dev), new=torch.empty(n_out, dtype=torch.int32, device=dev))
    g = gauss_struct(mu0, scale, quat, rho)
    _check(lib().digs_densify_apply(C.byref(g), _ptr(action), _ptr(dst), _ptr(_f32(z.contiguous(), "z")), n_out,
                                    _ptr(out["mu0"]), _ptr(out["scale"]), _ptr(out["quat"]), _ptr(out["rho"]),
                                    _ptr(out["src"]), _ptr(out["new"]), _stream()), "digs_densify_apply")
    return out


def gather_rows(src: torch.Tensor, new: torch.Tensor, rows: torch.Tensor) -> torch.Tensor:
    """rows [n][d] carried over to the densified cloud: the parent's row, zero for new rows."""
    rows = _f32(rows, "rows").contiguous()
    n_out, d = int(src.shape[0]), int(rows.shape[1]) if rows.dim() > 1 else 1
    out = torch.empty(n_out, d, device=rows.device)
    _check(lib().digs_gather_rows(_ptr(src), _ptr(new), n_out, d, _ptr(rows), _ptr(out), _stream()),
           "digs_gather_rows")
    return out


DIGS_CNN_TENSOR_CORES = 1


class WeightPredictor:
    """The weight-predictor CNN (include/digs.h, "Weight-predictor CNN"): parameters, Adam moments and
    a workspace in device memory; training and inference run in the library's kernels.  tensor_cores:
    the default of train_step (BF16-operand GEMMs on the tensor cores; False: FP32 SIMT)."""

    def __init__(self, R: int, seed: int = 0, input_scale: float = 1.0, device="cuda", tensor_cores: bool = True):
        self.tensor_cores = bool(tensor_cores)
        self.R = int(R)
        self.dev = torch.device(device)
        n = int(lib().digs_cnn_params(self.R))
        if n == 0:
            raise ValueError("unsupported R")
        self.params = torch.empty(n, device=self.dev)
        self.m = torch.zeros(n, device=self.dev)
        self.v = torch.zeros(n, device=self.dev)
        self.grad = torch.zeros(n, device=self.dev)
        self.step_count = 0
        self.input_scale = float(input_scale)
        self.loss = torch.zeros(1, device=self.dev)
        self.ws = Workspace(self.dev)
        _check(lib().digs_cnn_init(_ptr(self.params), self.R, int(seed), _stream()), "digs_cnn_init")

    def _ws(self, B: int):
        nb = int(lib().digs_cnn_workspace_size(B, self.R))
        if nb == 0:
            raise ValueError("batch size out of range")
        self.ws.ensure(nb)

    def prepare(self, proj: torch.Tensor) -> torch.Tensor:
        """[B][256][256] projections -> [B][128][128] network inputs (2x2 means times input_scale);
        [B][128][128] projections are only scaled."""
        proj = _f32(proj, "proj")
        B, nv, nu = proj.shape
        img = torch.empty(B, 128, 128, device=proj.device)
        _check(lib().digs_cnn_prepare_input(_ptr(proj), B, nu, nv, self.input_scale, _ptr(img), _stream()),
               "digs_cnn_prepare_input")
        return img

    def forward(self, img: torch.Tensor, cs: torch.Tensor, tensor_cores: bool = False) -> torch.Tensor:
        B = int(img.shape[0])
        self._ws(B)
        out = torch.empty(B, self.R, device=self.dev)
        flags = DIGS_CNN_TENSOR_CORES if tensor_cores else 0
        _check(lib().digs_cnn_forward(_ptr(self.params), self.R, _ptr(_f32(img, "img")), _ptr(_f32(cs, "cs")), B,
                                      _ptr(out), flags, self.ws.ptr, self.ws.nbytes, _stream()), "digs_cnn_forward")
        return out

    def backward(self, grad_w: torch.Tensor, tensor_cores: bool = False) -> torch.Tensor:
        """Parameter gradient for dL/dw of the preceding forward (same batch size)."""
        B = int(grad_w.shape[0])
        g = torch.empty_like(self.params)
        flags = DIGS_CNN_TENSOR_CORES if tensor_cores else 0
        _check(lib().digs_cnn_backward(_ptr(self.params), self.R, B, _ptr(_f32(grad_w, "grad_w")), _ptr(g), flags,
                                       self.ws.ptr, self.ws.nbytes, _stream()), "digs_cnn_backward")
        return g

    def train_step(self, img: torch.Tensor, cs: torch.Tensor, target: torch.Tensor, lr: float,
                   tensor_cores: Optional[bool] = None) -> torch.Tensor:
        B = int(img.shape[0])
        self._ws(B)
        self.step_count += 1
        tc = self.tensor_cores if tensor_cores is None else bool(tensor_cores)
        _check(lib().digs_cnn_train_step(_ptr(self.params), _ptr(self.m), _ptr(self.v), _ptr(self.grad),
                                         self.step_count, float(lr), self.R, _ptr(_f32(img, "img")),
                                         _ptr(_f32(cs, "cs")), _ptr(_f32(target, "target")), B, _ptr(self.loss),
                                         DIGS_CNN_TENSOR_CORES if tc else 0, self.ws.ptr, self.ws.nbytes,
                                         _stream()), "digs_cnn_train_step")
        return self.loss

    def predict(self, img: torch.Tensor, cs: torch.Tensor, batch: int = 512) -> torch.Tensor:
        """BF16-weight, FP32-accumulate inference in batches."""
        out = torch.empty(int(img.shape[0]), self.R, device=self.dev)
        for s in range(0, int(img.shape[0]), batch):
            B = min(batch, int(img.shape[0]) - s)
            self._ws(B)
            _check(lib().digs_cnn_infer_bf16(_ptr(self.params), self.R, _ptr(_f32(img[s:s + B], "img")),
                                             _ptr(_f32(cs[s:s + B], "cs")), B, _ptr(out[s:s + B]), self.ws.ptr,
                                             self.ws.nbytes, _stream()), "digs_cnn_infer_bf16")
        return out


class DigsGrid(C.Structure):
    _fields_ = [("nx", C.c_int), ("ny", C.c_int), ("nz", C.c_int), ("origin", C.c_float * 3),
                ("spacing", C.c_float * 3)]


def grid_struct(grid: Dict) -> DigsGrid:
    g = DigsGrid()
    g.nx, g.ny, g.nz = int(grid["nx"]), int(grid["ny"]), int(grid["nz"])
    for a in range(3):
        g.origin[a] = float(grid["origin"][a])
        g.spacing[a] = float(grid["spacing"][a])
    return g


def voxelize(mu0, scale, quat, rho, phi, w_row, lattice: Dict, grid: Dict, cutoff: float = 3.5) -> torch.Tensor:
    """Attenuation volume [nz][ny][nx] of the cloud deformed with weights w_row [R] (one time point)."""
    g = gauss_struct(mu0, scale, quat, rho)
    lat, gr = lattice_struct(lattice), grid_struct(grid)
    vol = torch.empty(gr.nz, gr.ny, gr.nx, device=mu0.device)
    o = opts_struct(cutoff)
    _check(lib().digs_voxelize(C.byref(g), C.byref(lat), _ptr(_f32(phi, "phi")), _ptr(_f32(w_row, "w")), C.byref(gr),
                               C.byref(o), _ptr(vol), _stream()), "digs_voxelize")
    return vol


def dvf(phi, w_row, lattice: Dict, grid: Dict) -> torch.Tensor:
    """Displacement field [nz][ny][nx][3] (mm) of one time point at the voxel centres."""
    lat, gr = lattice_struct(lattice), grid_struct(grid)
    out = torch.empty(gr.nz, gr.ny, gr.nx, 3, device=phi.device)
    _check(lib().digs_dvf(C.byref(lat), _ptr(_f32(phi, "phi")), _ptr(_f32(w_row, "w")), C.byref(gr), _ptr(out),
                          _stream()), "digs_dvf")
    return out
