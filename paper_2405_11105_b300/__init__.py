"""Python binding of the B300 localized EVD clutter filter (C ABI in include/lcf.h).

Argument marshalling only: every step of the filter runs in the CUDA library
``_lib/liblcf.so`` (sm_103a).  The functions keep the C names; ``Plan`` wraps
them for torch tensors (PyTorch provides device memory and streams).

There is no CPU fallback: if the library is missing, importing the binding
raises.
"""
from __future__ import annotations

import ctypes as C
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "_lib", "liblcf.so")

(LCF_OK, LCF_EINVAL, LCF_ENOMEM, LCF_ECUDA, LCF_ENOCONV, LCF_ETIMEOUT, LCF_EDEGENERATE, LCF_EUNSUPPORTED,
 LCF_ESCRATCH) = range(9)
(LCF_T_FIXED, LCF_T_CURVATURE, LCF_T_SLOPE, LCF_T_MEDIAN, LCF_T_SIGMOID, LCF_T_ADAPTIVE_SOFT,
 LCF_T_NONE, LCF_T_LEARNED, LCF_T_NCC) = range(9)
LCF_WFLAG_NOCONV, LCF_WFLAG_DEGENERATE, LCF_WFLAG_FALLBACK, LCF_WFLAG_SWEEP_SHIFT = 1, 2, 4, 8
LCF_PATH_SIMT, LCF_PATH_TC = 0, 1
LCF_EVD_CTA, LCF_EVD_PAIR, LCF_EVD_OS = 0, 1, 2
LCF_GP_F16X3, LCF_GP_BF16X3, LCF_GP_F16, LCF_GP_BF16, LCF_GP_E4M3 = range(5)
LCF_EP_FP32, LCF_EP_FP64_POLISH = 0, 1
LCF_PF_IDENTITY, LCF_PF_SUBTRACT = 0, 1
STAGES = ("prep", "gram", "assemble", "evd", "project")
EVD_PHASES = ("subspace", "qr", "congruence", "convert_q", "jacobi", "sort_phase", "rule", "weights")


class lcf_config(C.Structure):
    _fields_ = [("nz", C.c_int), ("nx", C.c_int), ("nt", C.c_int), ("wz", C.c_int), ("wx", C.c_int),
                ("sigma_scale", C.c_float), ("support_sigmas", C.c_float),
                ("all_ones_window", C.c_int), ("thresh_mode", C.c_int), ("beta", C.c_float),
                ("k_fixed", C.c_int), ("k_src", C.c_int), ("beta_src", C.c_float),
                ("pd_mode", C.c_int), ("alpha_mode", C.c_int), ("curv_norm", C.c_int),
                ("gram_path", C.c_int), ("project_path", C.c_int), ("max_sweeps", C.c_int),
                ("evd_path", C.c_int), ("inputs_ready", C.c_int),
                ("gram_precision", C.c_int), ("evd_precision", C.c_int), ("graph", C.c_int),
                ("project_form", C.c_int), ("deflate", C.c_int), ("inflight", C.c_int)]


class lcf_tuning(C.Structure):
    _fields_ = [("gram_splits", C.c_int), ("simt_gram_splits", C.c_int), ("aug_splits", C.c_int),
                ("q_splits", C.c_int), ("basis_splits", C.c_int), ("ncc_splits", C.c_int),
                ("evd_cluster", C.c_int)]

    def as_dict(self):
        return {f[0]: getattr(self, f[0]) for f in self._fields_}


class LcfError(RuntimeError):
    def __init__(self, status: int, where: str):
        super().__init__(f"{where}: {lcf_status_string(status)} (status {status})")
        self.status = status


def _load():
    if not os.path.exists(LIB_PATH):
        raise ImportError(f"CUDA library not built: {LIB_PATH} (run paper_2405_11105_b300/build.py)")
    L = C.CDLL(LIB_PATH)
    vp, ip, dp, fp = C.c_void_p, C.POINTER(C.c_int), C.POINTER(C.c_double), C.POINTER(C.c_float)
    sigs = {
        "lcf_config_default": ([C.POINTER(lcf_config), C.c_int, C.c_int, C.c_int, C.c_int, C.c_int], C.c_int),
        "lcf_plan_create": ([C.POINTER(lcf_config), C.c_int, C.POINTER(vp)], C.c_int),
        "lcf_filter": ([vp, vp, vp, vp], C.c_int),
        "lcf_filter_many": ([vp, vp, C.c_int, vp, vp], C.c_int),
        "lcf_filter_host": ([vp, vp, vp, vp], C.c_int),
        "lcf_filter_host_async": ([vp, vp, vp, vp], C.c_int),
        "lcf_plan_sync": ([vp], C.c_int),
        "lcf_filter_stream": ([vp, vp, C.c_int, C.c_int, vp, vp], C.c_int),
        "lcf_plan_status": ([vp, ip], C.c_int),
        "lcf_debug_dump": ([vp, dp, fp, ip, fp], C.c_int),
        "lcf_debug_gram": ([vp, dp], C.c_int),
        "lcf_debug_eigvecs": ([vp, fp], C.c_int),
        "lcf_debug_filtered_iq": ([vp, vp, C.c_int, vp, vp], C.c_int),
        "lcf_plan_windows": ([vp, ip, C.c_int, ip], C.c_int),
        "lcf_plan_workspace_bytes": ([vp], C.c_size_t),
        "lcf_plan_launch_count": ([vp, C.POINTER(C.c_longlong)], C.c_int),
        "lcf_plan_evd_phases": ([vp, dp], C.c_int),
        "lcf_plan_profile": ([vp, C.c_int], C.c_int),
        "lcf_plan_profile_read": ([vp, dp, ip], C.c_int),
        "lcf_plan_destroy": ([vp], C.c_int),
        "lcf_status_string": ([C.c_int], C.c_char_p),
        "lcf_gram_noalloc": ([C.POINTER(lcf_config), vp, vp, vp], C.c_int),
        "lcf_gram_noalloc_scratch_bytes": ([], C.c_size_t),
        "lcf_mlp_create": ([C.c_int, C.c_int, C.c_int, C.c_int, C.POINTER(vp)], C.c_int),
        "lcf_mlp_param_count": ([vp], C.c_size_t),
        "lcf_mlp_set_params": ([vp, fp], C.c_int),
        "lcf_mlp_get_params": ([vp, fp], C.c_int),
        "lcf_mlp_get_grads": ([vp, fp], C.c_int),
        "lcf_mlp_forward": ([vp, vp, C.c_int, vp, vp], C.c_int),
        "lcf_mlp_loss_grad": ([vp, vp, vp, C.c_int, fp, vp], C.c_int),
        "lcf_mlp_adamw": ([vp, C.c_float, C.c_float, C.c_float, C.c_float, C.c_float, vp], C.c_int),
        "lcf_mlp_destroy": ([vp], C.c_int),
        "lcf_plan_set_mlp": ([vp, vp, C.c_float], C.c_int),
        "lcf_debug_learned": ([vp, fp, fp], C.c_int),
        "lcf_plan_get_tuning": ([vp, C.POINTER(lcf_tuning)], C.c_int),
        "lcf_plan_set_tuning": ([vp, C.POINTER(lcf_tuning)], C.c_int),
        "lcf_plan_autotune": ([vp, vp, vp, C.c_char_p, ip], C.c_int),
        "lcf_selftest_wait_timeout": ([C.c_int, C.c_ulonglong, dp], C.c_int),
    }
    for name, (args, res) in sigs.items():
        f = getattr(L, name)
        f.argtypes = args
        f.restype = res
    return L


_lib = _load()

# ---- C-named wrappers (raw pointers as ints) ----


def lcf_status_string(s: int) -> str:
    return _lib.lcf_status_string(int(s)).decode()


def lcf_config_default(nz, nx, nt, wz, wx) -> lcf_config:
    c = lcf_config()
    _check(_lib.lcf_config_default(C.byref(c), nz, nx, nt, wz, wx), "lcf_config_default")
    return c


def lcf_plan_create(cfg: lcf_config, device: int = 0) -> int:
    h = C.c_void_p()
    _check(_lib.lcf_plan_create(C.byref(cfg), int(device), C.byref(h)), "lcf_plan_create")
    return h.value


def lcf_filter(plan: int, d_iq: int, d_out_pd: int, stream: int = 0) -> int:
    return _lib.lcf_filter(plan, d_iq, d_out_pd, stream)


def lcf_filter_host(plan: int, h_iq: int, h_out_pd: int, stream: int = 0) -> int:
    return _lib.lcf_filter_host(plan, h_iq, h_out_pd, stream)


def lcf_filter_host_async(plan: int, h_iq: int, h_out_pd: int, stream: int = 0) -> int:
    return _lib.lcf_filter_host_async(plan, h_iq, h_out_pd, stream)


def lcf_plan_sync(plan: int) -> int:
    return _lib.lcf_plan_sync(plan)


def lcf_filter_stream(plan: int, d_frames: int, n_frames: int, stride: int, d_out: int, stream: int = 0) -> int:
    return _lib.lcf_filter_stream(plan, d_frames, int(n_frames), int(stride), d_out, stream)


def lcf_plan_destroy(plan: int) -> int:
    return _lib.lcf_plan_destroy(plan)


def lcf_gram_noalloc(cfg: lcf_config, d_iq: int, d_R: int, stream: int = 0) -> int:
    """Windowed Gram matrices with no allocation (static per-device scratch)."""
    return _lib.lcf_gram_noalloc(C.byref(cfg), d_iq, d_R, stream)


def lcf_gram_noalloc_scratch_bytes() -> int:
    return int(_lib.lcf_gram_noalloc_scratch_bytes())


def _check(s: int, where: str):
    if s != LCF_OK:
        raise LcfError(s, where)


def _p(a, ct):
    return a.ctypes.data_as(C.POINTER(ct))


class Plan:
    """A filter plan on one device.  Tensors are torch tensors on that device."""

    def __init__(self, cfg: lcf_config, device: int = 0):
        self.cfg = cfg
        self.device = device
        self.handle = lcf_plan_create(cfg, device)
        nd = C.c_int()
        _check(_lib.lcf_plan_windows(self.handle, C.byref(nd), -1, None), "lcf_plan_windows")
        self.nd = nd.value

    @staticmethod
    def make(nz, nx, nt, wz, wx, device=0, **kw) -> "Plan":
        c = lcf_config_default(nz, nx, nt, wz, wx)
        for k, v in kw.items():
            if not hasattr(c, k):
                raise AttributeError(k)
            setattr(c, k, v)
        return Plan(c, device)

    def close(self):
        if self.handle:
            lcf_plan_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def evd_phases(self):
        """Mean SM cycles per EVD phase of the last call made while profiling was on."""
        cyc = np.zeros(len(EVD_PHASES))
        _check(_lib.lcf_plan_evd_phases(self.handle, _p(cyc, C.c_double)), "lcf_plan_evd_phases")
        return dict(zip(EVD_PHASES, cyc.tolist()))

    def set_mlp(self, mlp: "Mlp", p_min: float = 0.5):
        """Give the plan the learned cutoff rule (used when thresh_mode == LCF_T_LEARNED)."""
        _check(_lib.lcf_plan_set_mlp(self.handle, mlp.handle, float(p_min)), "lcf_plan_set_mlp")

    def tuning(self) -> lcf_tuning:
        """The plan's launch tuning (lcf_plan_get_tuning)."""
        t = lcf_tuning()
        _check(_lib.lcf_plan_get_tuning(self.handle, C.byref(t)), "lcf_plan_get_tuning")
        return t

    def set_tuning(self, **kw):
        """Change some tunables (lcf_plan_set_tuning); returns the new tuning."""
        t = self.tuning()
        for k, v in kw.items():
            if not hasattr(t, k):
                raise AttributeError(k)
            setattr(t, k, int(v))
        _check(_lib.lcf_plan_set_tuning(self.handle, C.byref(t)), "lcf_plan_set_tuning")
        return t

    def autotune(self, iq, cache_path=None, stream=None) -> bool:
        """Autotune the launch shapes on one packet (lcf_plan_autotune); True if the result
        came from the cache file."""
        import torch
        st = (stream or torch.cuda.current_stream(iq.device)).cuda_stream
        hit = C.c_int()
        path = None if cache_path is None else str(cache_path).encode()
        _check(_lib.lcf_plan_autotune(self.handle, iq.data_ptr(), st, path, C.byref(hit)), "lcf_plan_autotune")
        return bool(hit.value)

    def launch_count(self) -> int:
        """Kernels this plan has launched since it was created."""
        n = C.c_longlong()
        _check(_lib.lcf_plan_launch_count(self.handle, C.byref(n)), "lcf_plan_launch_count")
        return n.value

    @property
    def workspace_bytes(self) -> int:
        return int(_lib.lcf_plan_workspace_bytes(self.handle))

    def window_box(self, k: int):
        box = np.zeros(4, np.int32)
        _check(_lib.lcf_plan_windows(self.handle, None, int(k), _p(box, C.c_int)), "lcf_plan_windows")
        return tuple(int(v) for v in box)

    def filter(self, iq, out=None, stream=None):
        """iq: complex64 CUDA tensor [nt, nz, nx] -> float32 PD image [nz, nx]."""
        import torch
        c = self.cfg
        if iq.dtype != torch.complex64 or not iq.is_cuda or not iq.is_contiguous():
            raise ValueError("iq must be a contiguous complex64 CUDA tensor")
        if tuple(iq.shape) != (c.nt, c.nz, c.nx):
            raise ValueError(f"iq shape {tuple(iq.shape)} != {(c.nt, c.nz, c.nx)}")
        if out is None:
            out = torch.empty((c.nz, c.nx), dtype=torch.float32, device=iq.device)
        st = (stream or torch.cuda.current_stream(iq.device)).cuda_stream
        _check(lcf_filter(self.handle, iq.data_ptr(), out.data_ptr(), st), "lcf_filter")
        return out

    def filter_many(self, iq, out=None, stream=None):
        """iq: complex64 CUDA tensor [npk, nt, nz, nx] -> float32 PD images [npk, nz, nx]; up to
        cfg.inflight packets in progress at once (lcf_filter_many)."""
        import torch
        c = self.cfg
        if iq.dtype != torch.complex64 or not iq.is_cuda or not iq.is_contiguous():
            raise ValueError("iq must be a contiguous complex64 CUDA tensor")
        if iq.dim() != 4 or tuple(iq.shape[1:]) != (c.nt, c.nz, c.nx):
            raise ValueError(f"iq shape {tuple(iq.shape)} != (npk, {c.nt}, {c.nz}, {c.nx})")
        npk = iq.shape[0]
        if out is None:
            out = torch.empty((npk, c.nz, c.nx), dtype=torch.float32, device=iq.device)
        st = (stream or torch.cuda.current_stream(iq.device)).cuda_stream
        _check(_lib.lcf_filter_many(self.handle, iq.data_ptr(), int(npk), out.data_ptr(), st), "lcf_filter_many")
        return out

    def filter_host(self, iq_host, out_host=None, stream=None):
        """Host buffers (numpy or pinned torch CPU tensors); synchronises."""
        import torch
        c = self.cfg
        if out_host is None:
            out_host = np.empty((c.nz, c.nx), np.float32)
        ip = iq_host.data_ptr() if isinstance(iq_host, torch.Tensor) else iq_host.ctypes.data
        op = out_host.data_ptr() if isinstance(out_host, torch.Tensor) else out_host.ctypes.data
        st = (stream or torch.cuda.current_stream(self.device)).cuda_stream
        _check(lcf_filter_host(self.handle, ip, op, st), "lcf_filter_host")
        return out_host

    def filter_host_async(self, iq_host, out_host, stream=None):
        """Pipelined host call (pinned torch CPU tensors): returns at once; the next call's
        input copy overlaps this packet's kernels.  Inputs stay untouched and outputs unread
        until sync()."""
        import torch
        st = (stream or torch.cuda.current_stream(self.device)).cuda_stream
        _check(lcf_filter_host_async(self.handle, iq_host.data_ptr(), out_host.data_ptr(), st),
               "lcf_filter_host_async")
        return out_host

    def sync(self):
        _check(lcf_plan_sync(self.handle), "lcf_plan_sync")

    def filter_stream(self, frames, stride: int, out=None, stream=None):
        import torch
        c = self.cfg
        nf = frames.shape[0]
        npk = (nf - c.nt) // stride + 1
        if out is None:
            out = torch.empty((npk, c.nz, c.nx), dtype=torch.float32, device=frames.device)
        st = (stream or torch.cuda.current_stream(frames.device)).cuda_stream
        _check(lcf_filter_stream(self.handle, frames.data_ptr(), nf, stride, out.data_ptr(), st),
               "lcf_filter_stream")
        return out

    def profile(self, enable: bool = True):
        """Per-stage CUDA-event timing of subsequent filter calls (see lcf_plan_profile)."""
        _check(_lib.lcf_plan_profile(self.handle, int(bool(enable))), "lcf_plan_profile")

    def profile_read(self):
        """(dict stage -> summed ms, number of calls) since profiling was enabled."""
        ms = np.zeros(len(STAGES))
        n = C.c_int()
        _check(_lib.lcf_plan_profile_read(self.handle, _p(ms, C.c_double), C.byref(n)), "lcf_plan_profile_read")
        return dict(zip(STAGES, ms.tolist())), n.value

    def status(self):
        flags = np.zeros(self.nd, np.int32)
        s = _lib.lcf_plan_status(self.handle, _p(flags, C.c_int))
        return s, flags

    def debug(self):
        nd, nt = self.nd, self.cfg.nt
        lam = np.zeros((nd, nt)); wt = np.zeros((nd, nt), np.float32)
        k = np.zeros(nd, np.int32); al = np.zeros(nd, np.float32)
        _check(_lib.lcf_debug_dump(self.handle, _p(lam, C.c_double), _p(wt, C.c_float), _p(k, C.c_int),
                                   _p(al, C.c_float)), "lcf_debug_dump")
        return {"lam": lam, "wt": wt, "k": k, "alpha": al}

    def debug_learned(self):
        """(features [nd, nt+2], logits [nd, nt]) of the learned rule in the last call."""
        nd, nt = self.nd, self.cfg.nt
        f = np.zeros((nd, nt + 2), np.float32)
        z = np.zeros((nd, nt), np.float32)
        _check(_lib.lcf_debug_learned(self.handle, _p(f, C.c_float), _p(z, C.c_float)), "lcf_debug_learned")
        return f, z

    def debug_gram(self):
        nd, nt = self.nd, self.cfg.nt
        R = np.zeros((nd, nt, nt), np.complex128)
        _check(_lib.lcf_debug_gram(self.handle, R.ctypes.data_as(C.POINTER(C.c_double))), "lcf_debug_gram")
        return R

    def debug_eigvecs(self):
        nd, nt = self.nd, self.cfg.nt
        V = np.zeros((nd, nt, nt), np.complex64)
        _check(_lib.lcf_debug_eigvecs(self.handle, V.ctypes.data_as(C.POINTER(C.c_float))), "lcf_debug_eigvecs")
        return V

    def debug_filtered_iq(self, iq, subset: int, stream=None):
        import torch
        out = torch.empty_like(iq)
        st = (stream or torch.cuda.current_stream(iq.device)).cuda_stream
        _check(_lib.lcf_debug_filtered_iq(self.handle, iq.data_ptr(), int(subset), out.data_ptr(), st),
               "lcf_debug_filtered_iq")
        return out


def _stream_handle(stream):
    import torch
    st = stream if stream is not None else torch.cuda.current_stream()
    return st.cuda_stream


class Mlp:
    """The learned cutoff rule's network (see lcf_mlp_* in include/lcf.h).  Inputs
    and labels are torch tensors on the network's device."""

    def __init__(self, nt: int, hidden: int = 256, max_batch: int = 4096, device: int = 0):
        h = C.c_void_p()
        _check(_lib.lcf_mlp_create(int(nt), int(hidden), int(max_batch), int(device), C.byref(h)), "lcf_mlp_create")
        self.handle, self.nt, self.hidden, self.max_batch, self.device = h.value, nt, hidden, max_batch, device
        self.nparams = int(_lib.lcf_mlp_param_count(self.handle))

    def set_params(self, flat):
        a = np.ascontiguousarray(flat, dtype=np.float32)
        assert a.size == self.nparams
        _check(_lib.lcf_mlp_set_params(self.handle, _p(a, C.c_float)), "lcf_mlp_set_params")

    def params(self):
        a = np.empty(self.nparams, np.float32)
        _check(_lib.lcf_mlp_get_params(self.handle, _p(a, C.c_float)), "lcf_mlp_get_params")
        return a

    def grads(self):
        a = np.empty(self.nparams, np.float32)
        _check(_lib.lcf_mlp_get_grads(self.handle, _p(a, C.c_float)), "lcf_mlp_get_grads")
        return a

    def forward(self, x, stream=None):
        import torch
        x = x.contiguous()
        out = torch.empty((x.shape[0], self.nt), dtype=torch.float32, device=x.device)
        _check(_lib.lcf_mlp_forward(self.handle, x.data_ptr(), int(x.shape[0]), out.data_ptr(), _stream_handle(stream)),
               "lcf_mlp_forward")
        return out

    def loss_grad(self, x, k, stream=None) -> float:
        x, k = x.contiguous(), k.contiguous()
        loss = C.c_float()
        _check(_lib.lcf_mlp_loss_grad(self.handle, x.data_ptr(), k.data_ptr(), int(x.shape[0]), C.byref(loss),
                                      _stream_handle(stream)), "lcf_mlp_loss_grad")
        return float(loss.value)

    def adamw(self, lr, beta1=0.9, beta2=0.999, eps=1e-8, wd=0.0, stream=None):
        _check(_lib.lcf_mlp_adamw(self.handle, float(lr), float(beta1), float(beta2), float(eps), float(wd),
                                  _stream_handle(stream)), "lcf_mlp_adamw")

    def close(self):
        if self.handle:
            _lib.lcf_mlp_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def selftest_wait_timeout(limit_s: float = 0.05, device: int = 0):
    """Run the bounded-wait self-test kernel; returns (status, seconds waited)."""
    w = C.c_double()
    st = _lib.lcf_selftest_wait_timeout(int(device), int(limit_s * 1e9), C.byref(w))
    return st, w.value
