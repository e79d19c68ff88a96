"""Python binding of libgw, the GB300 hot path of the Matsubara-time GW cycle
(Chu et al., arXiv:1602.02313, Sec. III.B).

The binding only marshals arguments: every step runs in libgw's CUDA kernels
behind the C ABI declared in include/gw.h. PyTorch supplies device memory and
the stream. There is no CPU fallback: if libgw.so is missing or fails to load,
the first use of any entry point raises GwError.

Entry points keep the C names: gw_create/GW, green_tau, polarization,
tau_to_freq, screen, selfenergy, continue_, cpe_setup.
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libgw.so")

GW_OK, GW_EINVAL, GW_ENOMEM, GW_ECUDA, GW_ESINGULAR, GW_ENOCONV, GW_ETIMEOUT, GW_EUNSUPPORTED = 0, -1, -2, -3, -4, -5, -6, -7
GW_FP64, GW_FP16X2, GW_F32X2, GW_F32 = 0, 1, 3, 4
GW_BOSE, GW_FERMI = 0, 1
GW_TAU_TO_IW, GW_IW_TO_TAU, GW_TAU_TO_IW_CONT = 0, 1, 2
GW_PADE, GW_CPE = 0, 1
GW_TUNE_POL_SEG_CHUNKS, GW_TUNE_POL_PART_MB, GW_TUNE_WAIT_CYCLES, GW_TUNE_FAULT_STALL, GW_TUNE_POL_FORM = 0, 1, 2, 3, 4
PREC = {"fp64": GW_FP64, "fp16x2": GW_FP16X2}

_STATUS = {0: "GW_OK", -1: "GW_EINVAL", -2: "GW_ENOMEM", -3: "GW_ECUDA", -4: "GW_ESINGULAR",
           -5: "GW_ENOCONV", -6: "GW_ETIMEOUT", -7: "GW_EUNSUPPORTED"}

# Every symbol declared in include/gw.h.
EXPORTS = ["gw_create", "gw_destroy", "gw_sync", "gw_last_error", "gw_green_tau", "gw_polarization", "gw_polarization_many",
           "gw_tau_to_freq", "gw_tau_to_freq_many", "gw_screen", "gw_screen_tau", "gw_dyson_tau", "gw_sigma_star", "gw_selfenergy_offdiag", "gw_dyson_matrix", "gw_selfenergy", "gw_continue", "gw_cpe_setup",
           "gw_cpe_coeffs", "gw_copy_m", "gw_transform_matrices", "gw_launch_count",
           "gw_kernel_timing", "gw_kernel_time", "gw_set_stream", "gw_set_tuning", "gw_measure_alu",
           "gw_screen_static", "gw_mlp_create", "gw_mlp_destroy", "gw_mlp_last_error", "gw_mlp_num_params",
           "gw_mlp_forward", "gw_mlp_loss_grad", "gw_mlp_train_step", "gw_mlp_sync", "gw_mlp_get_params", "gw_mlp_set_params",
           "gw_cpe_features", "gw_cpe_fit_matrix", "gw_cpe_seed", "gw_cpe_iterations"]


class GwError(RuntimeError):
    pass


class _Grid(ctypes.Structure):
    _fields_ = [("beta", ctypes.c_double), ("ntau", ctypes.c_int), ("tau", ctypes.POINTER(ctypes.c_double)),
                ("npole", ctypes.c_int), ("poles", ctypes.POINTER(ctypes.c_double)),
                ("nnu", ctypes.c_int), ("nu_idx", ctypes.POINTER(ctypes.c_int)),
                ("nw", ctypes.c_int), ("w_idx", ctypes.POINTER(ctypes.c_int)), ("ncont", ctypes.c_int)]


class _System(ctypes.Structure):
    _fields_ = [("seed", ctypes.c_uint64), ("nk", ctypes.c_int), ("nq", ctypes.c_int), ("nb", ctypes.c_int),
                ("nocc", ctypes.c_int), ("ni", ctypes.c_int), ("omega", ctypes.c_double),
                ("kmq", ctypes.POINTER(ctypes.c_int)), ("v", ctypes.POINTER(ctypes.c_double)),
                ("M", ctypes.c_void_p), ("q0", ctypes.c_int), ("m_mode", ctypes.c_int)]


def _grid_struct(grid, keep):
    """gw_grid view of a gwinputs.Grid-like object; `keep` holds the host arrays alive."""
    dp = ctypes.POINTER(ctypes.c_double)
    ip = ctypes.POINTER(ctypes.c_int)
    keep["tau"] = np.ascontiguousarray(grid.tau, np.float64)
    keep["poles"] = np.ascontiguousarray(grid.poles, np.float64)
    keep["nu"] = np.ascontiguousarray(grid.nu_idx, np.int32)
    keep["w"] = np.ascontiguousarray(grid.w_idx, np.int32)
    return _Grid(float(grid.beta), len(keep["tau"]), keep["tau"].ctypes.data_as(dp), len(keep["poles"]),
                 keep["poles"].ctypes.data_as(dp), len(keep["nu"]), keep["nu"].ctypes.data_as(ip),
                 len(keep["w"]), keep["w"].ctypes.data_as(ip), int(grid.ncont))


def measure_alu(device=0):
    """Measured (FP64 TFLOP/s, FP32 TFLOP/s) FMA throughput of `device`'s CUDA cores."""
    a, b = ctypes.c_double(), ctypes.c_double()
    st = lib().gw_measure_alu(int(device), ctypes.byref(a), ctypes.byref(b))
    if st != GW_OK:
        raise GwError(f"gw_measure_alu: {_STATUS.get(st, st)}")
    return a.value, b.value


def transform_matrices(grid):
    """Host-only: the transform matrices libgw builds for this grid (gw_transform_matrices)."""
    keep = {}
    g = _grid_struct(grid, keep)
    nt, nnu, nw, nc = g.ntau, g.nnu, g.nw, g.ncont
    bf = np.zeros((nnu, nt, 2))
    ff = np.zeros((nw, nt, 2))
    fc = np.zeros((nc, nt, 2))
    bb = np.zeros((nt, 2 * nnu))
    fb = np.zeros((nt, 2 * nw))
    dp = ctypes.c_void_p
    st = lib().gw_transform_matrices(ctypes.byref(g), dp(bf.ctypes.data), dp(ff.ctypes.data), dp(fc.ctypes.data),
                                     dp(bb.ctypes.data), dp(fb.ctypes.data))
    if st != GW_OK:
        raise GwError(f"gw_transform_matrices: {_STATUS.get(st, st)}")
    c = lambda a: a[..., 0] + 1j * a[..., 1]  # noqa: E731
    return {"B_fwd": c(bf), "F_fwd": c(ff), "F_cont": c(fc), "B_bwd_re": bb[:, :nnu], "B_bwd_im": bb[:, nnu:],
            "F_bwd_re": fb[:, :nw], "F_bwd_im": fb[:, nw:]}


def polarization_many(ctxs, iqs, Gs, Ps, prec=GW_FP16X2):
    """gw_polarization_many: the polarization of several contexts (one q each) in one persistent
    launch on ctxs[0]'s stream. ctxs: GW objects; iqs: q indices; Gs, Ps: device tensors."""
    n = len(ctxs)
    H = (ctypes.c_void_p * n)(*[c.h for c in ctxs])
    Q = (ctypes.c_int * n)(*[int(q) for q in iqs])
    G = (ctypes.c_void_p * n)(*[_ptr(g).value for g in Gs])
    P = (ctypes.c_void_p * n)(*[_ptr(p).value for p in Ps])
    st = lib().gw_polarization_many(n, H, Q, G, P, int(prec))
    if st != GW_OK:
        msg = lib().gw_last_error(ctxs[0].h)
        raise GwError(f"gw_polarization_many: {_STATUS.get(st, st)}: {msg.decode() if msg else ''}")


def load_library(path=LIB_PATH):
    """Load libgw.so and declare argument types; raises if it is missing."""
    if not os.path.exists(path):
        raise GwError(f"libgw.so not built at {path}: run __graft_entry__.build() (no CPU fallback)")
    lib = ctypes.CDLL(path)
    vp, i32, i64, dbl = ctypes.c_void_p, ctypes.c_int, ctypes.c_int64, ctypes.c_double
    sig = {
        "gw_create": [ctypes.POINTER(vp), ctypes.POINTER(_Grid), ctypes.POINTER(_System), i32, vp],
        "gw_destroy": [vp], "gw_sync": [vp], "gw_last_error": [vp],
        "gw_green_tau": [vp, vp, vp, vp, vp, vp, vp],
        "gw_polarization": [vp, i32, vp, i32, vp],
        "gw_polarization_many": [i32, vp, vp, vp, vp, i32],
        "gw_tau_to_freq": [vp, i32, i32, i64, vp, i32, vp],
        "gw_tau_to_freq_many": [vp, i32, i32, i32, i64, vp, i32, vp],
        "gw_screen_tau": [vp, i32, i32, vp, vp, vp, vp],
        "gw_dyson_tau": [vp, i64, i32, vp, vp, vp, vp, vp, vp],
        "gw_sigma_star": [vp, i32, vp, i64, vp, vp],
        "gw_selfenergy_offdiag": [vp, i32, vp, vp, vp, vp, vp],
        "gw_dyson_matrix": [vp, vp, vp, vp, vp, vp, vp, vp],
        "gw_screen": [vp, i32, i32, vp, i32, vp, vp],
        "gw_selfenergy": [vp, i32, vp, vp, vp, i32, vp, vp],
        "gw_continue": [vp, i32, i64, vp, vp, vp, vp, i32, vp, vp, vp, vp],
        "gw_cpe_setup": [vp, i32, ctypes.POINTER(dbl), dbl],
        "gw_cpe_coeffs": [vp, vp],
        "gw_copy_m": [vp, i32, i32, i32, vp],
        "gw_transform_matrices": [ctypes.POINTER(_Grid), vp, vp, vp, vp, vp],
        "gw_launch_count": [vp],
        "gw_kernel_timing": [vp, i32],
        "gw_set_stream": [vp, vp],
        "gw_set_tuning": [vp, i32, i64],
        "gw_measure_alu": [i32, vp, vp],
        "gw_kernel_time": [vp, ctypes.c_char_p, vp, vp],
        "gw_screen_static": [i32, i32, i32, vp, vp, vp, vp, vp],
        "gw_mlp_create": [ctypes.POINTER(vp), i32, i32, i32, i32, ctypes.c_uint64, i32, vp],
        "gw_mlp_destroy": [vp], "gw_mlp_last_error": [vp], "gw_mlp_num_params": [vp],
        "gw_mlp_forward": [vp, i64, vp, vp],
        "gw_mlp_loss_grad": [vp, i64, vp, i32, vp, vp, vp],
        "gw_mlp_train_step": [vp, i64, vp, i32, vp, ctypes.c_float, vp],
        "gw_mlp_get_params": [vp, vp], "gw_mlp_set_params": [vp, vp], "gw_mlp_sync": [vp],
        "gw_cpe_features": [vp, i64, vp, i32, vp, vp],
        "gw_cpe_fit_matrix": [vp, i32, vp],
        "gw_cpe_seed": [vp, i64, vp, vp],
        "gw_cpe_iterations": [vp, vp],
    }
    for name, args in sig.items():
        f = getattr(lib, name)
        f.argtypes = args
        f.restype = {"gw_last_error": ctypes.c_char_p, "gw_mlp_last_error": ctypes.c_char_p,
                     "gw_launch_count": ctypes.c_int64, "gw_mlp_num_params": ctypes.c_int64}.get(name, ctypes.c_int)
    return lib


_lib = None


def lib():
    global _lib
    if _lib is None:
        _lib = load_library()
    return _lib


def _ptr(t):
    """Device pointer of a contiguous CUDA tensor (or None -> NULL)."""
    if t is None:
        return None
    import torch
    if not isinstance(t, torch.Tensor) or not t.is_cuda:
        raise GwError("expected a CUDA tensor")
    if not t.is_contiguous():
        raise GwError("expected a contiguous tensor")
    return ctypes.c_void_p(t.data_ptr())


class GW:
    """A libgw context (gw_create / gw_destroy) bound to a torch CUDA stream.

    grid: gwinputs.Grid-like object (beta, tau, poles, nu_idx, w_idx, ncont)
    crystal: gwinputs.Crystal-like object (seed, nk, nq, nb, nocc, ni, v, kmq)
    omega: unit-cell volume in 1/(Omega N_k).
    """

    def __init__(self, grid, crystal, omega=1.0, device=0, stream=None, M=None, q0=0, m_mode=0):
        import torch
        self.lib = lib()
        self.device = device
        self.stream = stream if stream is not None else torch.cuda.current_stream(device)
        self.grid = grid
        self.cr = crystal
        self.omega = float(omega)
        self._h = {"kmq": np.ascontiguousarray(crystal.kmq, np.int32),
                   "v": np.ascontiguousarray(crystal.v, np.float64)}
        dp = ctypes.POINTER(ctypes.c_double)
        ip = ctypes.POINTER(ctypes.c_int)
        g = _grid_struct(grid, self._h)
        s = _System(int(crystal.seed), crystal.nk, crystal.nq, crystal.nb, crystal.nocc, crystal.ni, self.omega,
                    self._h["kmq"].ctypes.data_as(ip), self._h["v"].ctypes.data_as(dp),
                    None if M is None else ctypes.c_void_p(M.data_ptr()), int(q0), int(m_mode))
        self._M = M
        h = ctypes.c_void_p()
        with torch.cuda.device(device):
            st = self.lib.gw_create(ctypes.byref(h), ctypes.byref(g), ctypes.byref(s), device,
                                    ctypes.c_void_p(self.stream.cuda_stream))
        if st != GW_OK:
            raise GwError(f"gw_create failed: {_STATUS.get(st, st)}")
        self.h = h

    # ------------------------------------------------------------------
    def _check(self, st, what):
        if st != GW_OK:
            msg = self.lib.gw_last_error(self.h)
            raise GwError(f"{what}: {_STATUS.get(st, st)}: {msg.decode() if msg else ''}")

    def close(self):
        if getattr(self, "h", None):
            self.lib.gw_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def launch_count(self):
        return int(self.lib.gw_launch_count(self.h))

    def set_stream(self, stream):
        """Queue the following calls on `stream` (a torch.cuda.Stream on the context's device)."""
        self._check(self.lib.gw_set_stream(self.h, ctypes.c_void_p(stream.cuda_stream)), "gw_set_stream")
        self.stream = stream

    def set_tuning(self, key, value):
        self._check(self.lib.gw_set_tuning(self.h, int(key), int(value)), "gw_set_tuning")

    def kernel_timing(self, enable=True):
        """Record CUDA events around the tensor-core and screening launches from now on."""
        self._check(self.lib.gw_kernel_timing(self.h, int(bool(enable))), "gw_kernel_timing")

    def kernel_time(self, name):
        """(summed device ms, launches) of the named kernel since kernel_timing(True)."""
        ms, n = ctypes.c_double(), ctypes.c_int64()
        self._check(self.lib.gw_kernel_time(self.h, name.encode(), ctypes.byref(ms), ctypes.byref(n)),
                    "gw_kernel_time")
        return float(ms.value), int(n.value)

    def sync(self):
        self._check(self.lib.gw_sync(self.h), "gw_sync")

    # ------------------------------------------------------------------
    def green_tau(self, eps, G, occ, sigx=None, vxc=None, sigc_iw=None):
        self._check(self.lib.gw_green_tau(self.h, _ptr(eps), _ptr(sigx), _ptr(vxc), _ptr(sigc_iw), _ptr(G),
                                          _ptr(occ)), "gw_green_tau")

    def polarization(self, iq, G, P, prec=GW_FP64):
        self._check(self.lib.gw_polarization(self.h, iq, _ptr(G), int(prec), _ptr(P)), "gw_polarization")

    def tau_to_freq(self, stat, direction, batch, x, y, prec=GW_FP64):
        self._check(self.lib.gw_tau_to_freq(self.h, int(stat), int(direction), int(batch), _ptr(x), int(prec),
                                            _ptr(y)), "gw_tau_to_freq")

    def tau_to_freq_many(self, stat, direction, count, batch, x, y, prec=GW_FP64):
        self._check(self.lib.gw_tau_to_freq_many(self.h, int(stat), int(direction), int(count), int(batch), _ptr(x),
                                                 int(prec), _ptr(y)), "gw_tau_to_freq_many")

    def screen_tau(self, iq, tau, P_pair, Wt_tau, info):
        """tau: host float64 array (the mesh); P_pair, Wt_tau, info: device tensors."""
        t = np.ascontiguousarray(tau, dtype=np.float64)
        self._check(self.lib.gw_screen_tau(self.h, int(iq), int(t.size), ctypes.c_void_p(t.ctypes.data), _ptr(P_pair),
                                           _ptr(Wt_tau), _ptr(info)), "gw_screen_tau")

    def dyson_tau(self, tau_upm, eps, s, sigc, G, info):
        """tau_upm: host float64 mesh; eps, s [nprob], sigc [nprob][n_upm], G [nprob][n + 1], info: device."""
        t = np.ascontiguousarray(tau_upm, dtype=np.float64)
        self._check(self.lib.gw_dyson_tau(self.h, int(eps.numel()), int(t.size), ctypes.c_void_p(t.ctypes.data),
                                          _ptr(eps), _ptr(s), _ptr(sigc), _ptr(G), _ptr(info)), "gw_dyson_tau")

    def sigma_star(self, kinv, T, S):
        """kinv: device int32 [nrep][nk]; T, S: device float64 [nk][...] (S accumulated)."""
        self._check(self.lib.gw_sigma_star(self.h, int(kinv.shape[0]), _ptr(kinv), int(T.numel() // T.shape[0]),
                                           _ptr(T), _ptr(S)), "gw_sigma_star")

    def selfenergy_offdiag(self, iq, G, occ, W, S, Sx=None):
        """S: complex128 [nk][nb][nb][ntau], Sx: complex128 [nk][nb][nb] or None (both accumulated)."""
        self._check(self.lib.gw_selfenergy_offdiag(self.h, int(iq), _ptr(G), _ptr(occ), _ptr(W), _ptr(S), _ptr(Sx)),
                    "gw_selfenergy_offdiag")

    def dyson_matrix(self, eps, Sx, vxc, Sc_tau, G, occ, info):
        """Full-matrix Dyson update: eps [nk][nb]; Sx, vxc complex128 [nk][nb][nb] or None; Sc_tau
        complex128 [nk][nb][nb][ntau] or None; G complex128 [nk][nb][nb][ntau], occ complex128
        [nk][nb][nb], info int32 [nk] (outputs)."""
        self._check(self.lib.gw_dyson_matrix(self.h, _ptr(eps), _ptr(Sx), _ptr(vxc), _ptr(Sc_tau), _ptr(G), _ptr(occ),
                                             _ptr(info)), "gw_dyson_matrix")

    def screen(self, iq0, nqb, P_iv, W_iv, info, prec=GW_FP64):
        self._check(self.lib.gw_screen(self.h, iq0, nqb, _ptr(P_iv), int(prec), _ptr(W_iv), _ptr(info)), "gw_screen")

    def selfenergy(self, iq, G, occ, W_tau, S, Sx=None, prec=GW_FP64):
        self._check(self.lib.gw_selfenergy(self.h, iq, _ptr(G), _ptr(occ), _ptr(W_tau), int(prec), _ptr(S),
                                           _ptr(Sx)), "gw_selfenergy")

    def cpe_setup(self, x, ridge):
        x = np.ascontiguousarray(x, np.float64)
        self._check(self.lib.gw_cpe_setup(self.h, len(x) - 2, x.ctypes.data_as(ctypes.POINTER(ctypes.c_double)),
                                          float(ridge)), "gw_cpe_setup")

    def cpe_coeffs(self, b):
        self._check(self.lib.gw_cpe_coeffs(self.h, _ptr(b)), "gw_cpe_coeffs")

    def continue_(self, method, sig_iw, eps, sigx, vxc, omega_real, sig_real, e_qp, info):
        nprob = eps.numel()
        nreal = 0 if omega_real is None else omega_real.numel()
        self._check(self.lib.gw_continue(self.h, int(method), nprob, _ptr(sig_iw), _ptr(eps), _ptr(sigx),
                                         _ptr(vxc), nreal, _ptr(omega_real), _ptr(sig_real), _ptr(e_qp),
                                         _ptr(info)), "gw_continue")

    def copy_m(self, iq, k0, nkc, out):
        self._check(self.lib.gw_copy_m(self.h, iq, k0, nkc, _ptr(out)), "gw_copy_m")

    # ------------------------------------------------------------------ learned CPE seed
    def cpe_features(self, sig_iw, nfit, x, scale):
        self._check(self.lib.gw_cpe_features(self.h, scale.numel(), _ptr(sig_iw), int(nfit), _ptr(x), _ptr(scale)),
                    "gw_cpe_features")

    def cpe_fit_matrix(self, nfit, A):
        self._check(self.lib.gw_cpe_fit_matrix(self.h, int(nfit), _ptr(A)), "gw_cpe_fit_matrix")

    def cpe_seed(self, bhat, scale):
        self._check(self.lib.gw_cpe_seed(self.h, scale.numel(), _ptr(bhat), _ptr(scale)), "gw_cpe_seed")

    def cpe_iterations(self, iters):
        self._check(self.lib.gw_cpe_iterations(self.h, _ptr(iters)), "gw_cpe_iterations")


class MLP:
    """gw_mlp handle: the learned CPE seed network (tensor-core forward / backward / Adam)."""

    def __init__(self, nin=128, nh=256, nhidden=3, nout=128, seed=1, device=0, stream=None):
        import torch
        self.lib = lib()
        self.stream = stream if stream is not None else torch.cuda.current_stream(device)
        h = ctypes.c_void_p()
        st = self.lib.gw_mlp_create(ctypes.byref(h), nin, nh, nhidden, nout, seed, device,
                                    ctypes.c_void_p(self.stream.cuda_stream))
        if st != GW_OK:
            raise GwError(f"gw_mlp_create failed: {_STATUS.get(st, st)}")
        self.h = h
        self.nin, self.nout = nin, nout

    def _check(self, st, what):
        if st != GW_OK:
            msg = self.lib.gw_mlp_last_error(self.h)
            raise GwError(f"{what}: {_STATUS.get(st, st)}: {msg.decode() if msg else ''}")

    def close(self):
        if getattr(self, "h", None):
            self.lib.gw_mlp_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def num_params(self):
        return int(self.lib.gw_mlp_num_params(self.h))

    def forward(self, x, out):
        self._check(self.lib.gw_mlp_forward(self.h, x.shape[0], _ptr(x), _ptr(out)), "gw_mlp_forward")

    def loss_grad(self, x, A, loss=None, grads=None):
        self._check(self.lib.gw_mlp_loss_grad(self.h, x.shape[0], _ptr(x), x.shape[1], _ptr(A), _ptr(loss),
                                              _ptr(grads)), "gw_mlp_loss_grad")

    def train_step(self, x, A, lr, loss=None):
        self._check(self.lib.gw_mlp_train_step(self.h, x.shape[0], _ptr(x), x.shape[1], _ptr(A), float(lr),
                                               _ptr(loss)), "gw_mlp_train_step")

    def sync(self):
        self._check(self.lib.gw_mlp_sync(self.h), "gw_mlp_sync")

    def get_params(self):
        p = np.zeros(self.num_params(), np.float32)
        self._check(self.lib.gw_mlp_get_params(self.h, ctypes.c_void_p(p.ctypes.data)), "gw_mlp_get_params")
        return p

    def set_params(self, p):
        p = np.ascontiguousarray(p, np.float32)
        self._check(self.lib.gw_mlp_set_params(self.h, ctypes.c_void_p(p.ctypes.data)), "gw_mlp_set_params")
