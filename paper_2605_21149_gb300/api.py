"""Python binding of libqmlgb: argument marshalling only.

Every numeric step runs in the library's CUDA kernels; this module turns
torch tensors (device memory, current stream) or numpy arrays (host memory,
staged by the library) into the pointers and sizes of the C ABI.

Layout (see include/qmlgb.h): matrices are column-major.  A torch matrix of
shape (rows, cols) is used as-is when its strides are (1, rows) (e.g. the
transpose of a contiguous (cols, rows) tensor); otherwise a column-major copy
is made first.  Returned matrices are column-major views of that kind.
"""
from __future__ import annotations

import ctypes

import numpy as np

from . import _native as nat

try:
    import torch
except ImportError:  # pragma: no cover - torch is part of the supported setup
    torch = None


BASIS_PIXEL, BASIS_HARMONIC, BASIS_AUTO = (nat.QML_BASIS_PIXEL, nat.QML_BASIS_HARMONIC,
                                           nat.QML_BASIS_AUTO)


class QMLError(RuntimeError):
    def __init__(self, status: int, msg: str):
        super().__init__(f"{nat.STATUS_NAMES.get(status, status)}: {msg}")
        self.status = status


def _lib():
    return nat.load()


def _check(status: int):
    if status != nat.QML_OK:
        raise QMLError(status, _lib().qml_last_error().decode(errors="replace"))


def _is_torch(x):
    return torch is not None and isinstance(x, torch.Tensor)


def _stream(device_mode: bool):
    if device_mode and torch is not None and torch.cuda.is_available():
        return ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    return ctypes.c_void_p(0)


def _vec(x, keep):
    """float64 contiguous vector -> pointer (kept alive in `keep`)."""
    if x is None:
        return None
    if _is_torch(x):
        t = x.to(torch.float64).contiguous()
        keep.append(t)
        return t.data_ptr()
    a = np.ascontiguousarray(x, dtype=np.float64)
    keep.append(a)
    return a.ctypes.data


def _mat(x, rows, cols, keep):
    """float64 column-major (rows x cols) -> pointer."""
    if _is_torch(x):
        t = x.to(torch.float64)
        if t.dim() == 1:
            t = t.reshape(rows, cols) if cols == 1 else t.reshape(cols, rows).t()
        if not (t.shape == (rows, cols) and (t.stride() == (1, rows) or cols == 1 and t.is_contiguous())):
            t = t.reshape(rows, cols).t().contiguous().t()
        keep.append(t)
        return t.data_ptr()
    a = np.asarray(x, dtype=np.float64)
    a = np.asfortranarray(a.reshape(rows, cols) if a.ndim == 1 else a)
    assert a.shape == (rows, cols), (a.shape, rows, cols)
    keep.append(a)
    return a.ctypes.data


def _empty(rows, cols, like_device):
    """Column-major (rows x cols) output: torch on the device or numpy on the host."""
    if like_device:
        return torch.empty((cols, rows), dtype=torch.float64, device="cuda").t()
    return np.empty((rows, cols), dtype=np.float64, order="F")


def _ptr(x):
    return x.data_ptr() if _is_torch(x) else x.ctypes.data


SPEC_INDEX = {"TT": 0, "EE": 1, "BB": 2, "TE": 3, "TB": 4, "EB": 5}


class Problem:
    """One analysis: geometry, band, transfer, spectra, noise (qml_problem).

    Arrays may be torch tensors (device mode: everything must be on the GPU)
    or numpy arrays (host mode: the library copies them in and results out).
    """

    def __init__(self, lmin, lmax, *, theta_T=None, phi_T=None, theta_P=None, phi_P=None,
                 transfer_T=None, transfer_P=None, spec=("TT",), cl_fid=None, N=None,
                 precision=nat.QML_FP64, nslices=0, bin_edges=None, lsig=None,
                 basis=nat.QML_BASIS_PIXEL):
        self._keep = []
        has_T = theta_T is not None
        has_P = theta_P is not None
        probe = next(a for a in (theta_T, theta_P) if a is not None)
        self.device = _is_torch(probe)
        self.lmin, self.lmax = int(lmin), int(lmax)
        self.npix_T = len(theta_T) if has_T else 0
        self.npix_P = len(theta_P) if has_P else 0
        self.n = self.npix_T + 2 * self.npix_P
        self.comps = ((0,) if has_T else ()) + ((1, 2) if has_P else ())
        self.k0 = (self.lmax + 1) ** 2 - self.lmin ** 2
        self.k = len(self.comps) * self.k0
        self.nl = self.lmax - self.lmin + 1
        self.spec = tuple(SPEC_INDEX[s] if isinstance(s, str) else int(s) for s in spec)
        # native binning (Sect. 2.4): host edges lmin = e_0 < ... < e_nb = lmax + 1
        edges = None if bin_edges is None else np.ascontiguousarray(bin_edges, dtype=np.int32)
        self.nb = self.nl if edges is None else len(edges) - 1
        self.na = len(self.spec) * self.nb
        p = nat.QmlProblem()
        p.has_T, p.has_P = int(has_T), int(has_P)
        p.npix_T, p.npix_P = self.npix_T, self.npix_P
        p.theta_T, p.phi_T = _vec(theta_T, self._keep), _vec(phi_T, self._keep)
        p.theta_P, p.phi_P = _vec(theta_P, self._keep), _vec(phi_P, self._keep)
        p.lmin, p.lmax = self.lmin, self.lmax
        p.transfer_T = _vec(transfer_T, self._keep)
        p.transfer_P = _vec(transfer_P, self._keep)
        p.nspec = len(self.spec)
        for i, s in enumerate(self.spec):
            p.spec[i] = s
        p.cl_fid = _vec(cl_fid, self._keep) if cl_fid is not None else None
        p.N = _mat(N, self.n, self.n, self._keep) if N is not None else None
        p.precision = int(precision)
        p.nslices = int(nslices)
        # multipole switching: signal band (lmin_sig, lmax_sig) around the window;
        # transfer and cl_fid then cover it (cl_fid is [6][lmax_sig + 1])
        if lsig is not None:
            p.lmin_sig, p.lmax_sig = int(lsig[0]), int(lsig[1])
        p.basis = int(basis)
        if edges is not None:
            self._keep.append(edges)
            p.nbins = len(edges) - 1
            p.bin_edges = edges.ctypes.data
        self._p = p

    @classmethod
    def from_workload(cls, wl, device=True, precision=nat.QML_FP64, nslices=0, bin_edges=None,
                      window=None, basis=nat.QML_BASIS_PIXEL):
        """Problem from a synth.Workload; device=True puts every array on cuda:0.
        window=(lmin, lmax) inside the workload's band estimates only that
        window, the workload's band being the signal band (multipole switching)."""
        def conv(a):
            if a is None or len(a) == 0:
                return None
            if device:
                return torch.as_tensor(np.ascontiguousarray(a), dtype=torch.float64, device="cuda")
            return np.ascontiguousarray(a, dtype=np.float64)
        N = wl.N()
        lmin, lmax = (wl.lmin, wl.lmax) if window is None else window
        lsig = None if window is None else (wl.lmin, wl.lmax)
        return cls(lmin, lmax,
                   theta_T=conv(wl.theta_T) if wl.has_T else None,
                   phi_T=conv(wl.phi_T) if wl.has_T else None,
                   theta_P=conv(wl.theta_P) if wl.has_P else None,
                   phi_P=conv(wl.phi_P) if wl.has_P else None,
                   transfer_T=conv(wl.transfer_T) if wl.has_T else None,
                   transfer_P=conv(wl.transfer_P) if wl.has_P else None,
                   spec=wl.spec, cl_fid=conv(wl.cl_fid.reshape(-1)),
                   N=(torch.as_tensor(N, device="cuda") if device else N),
                   precision=precision, nslices=nslices, bin_edges=bin_edges, lsig=lsig,
                   basis=basis)

    @property
    def ref(self):
        return ctypes.byref(self._p)


def ybuild(prob: Problem):
    """Y (n x k, column-major), transfer folded in (qml_ybuild)."""
    Y = _empty(prob.n, prob.k, prob.device)
    _check(_lib().qml_ybuild(prob.ref, _ptr(Y), prob.n, _stream(prob.device)))
    return Y


def synthesize(prob: Problem, alm, noise):
    """maps = Y alm + noise (qml_synthesize); alm k x nsims, noise n x nsims."""
    keep = []
    nsims = alm.shape[1] if alm.ndim == 2 else 1
    a = _mat(alm, prob.k, nsims, keep)
    nz = _mat(noise, prob.n, nsims, keep)
    out = _empty(prob.n, nsims, prob.device)
    _check(_lib().qml_synthesize(prob.ref, a, nz, nsims, _ptr(out), _stream(prob.device)))
    return out


class Plan:
    """Fisher-stage state reused by the estimates (qml_plan)."""

    def __init__(self, handle, prob: Problem):
        self._h = handle
        self.prob = prob

    def estimate(self, maps):
        """dict y, b, cl_deconv, cl_decorr, q_conv for the columns of maps (n x nsims)."""
        keep = []
        pr = self.prob
        nsims = maps.shape[1] if maps.ndim == 2 else 1
        d = _mat(maps, pr.n, nsims, keep)
        dev = pr.device
        out = {k: _empty(pr.na, nsims, dev) for k in ("y", "cl_deconv", "cl_decorr", "q_conv")}
        out["b"] = _empty(pr.na, 1, dev)
        _check(_lib().qml_estimate(self._h, d, nsims, _ptr(out["y"]), _ptr(out["b"]),
                                   _ptr(out["cl_deconv"]), _ptr(out["cl_decorr"]),
                                   _ptr(out["q_conv"]), _stream(dev)))
        out["b"] = out["b"][:, 0]
        return out

    @property
    def basis(self):
        """QML_BASIS_PIXEL or QML_BASIS_HARMONIC: the basis qml_fisher used."""
        return _lib().qml_plan_basis(self._h)

    def free(self):
        if self._h:
            _lib().qml_plan_free(self._h)
            self._h = None

    def __del__(self):
        try:
            self.free()
        except Exception:
            pass


def fisher(prob: Problem, keep_plan: bool = True):
    """(F, plan) from qml_fisher; F is na x na, spectrum-major."""
    F = _empty(prob.na, prob.na, prob.device)
    h = ctypes.c_void_p(0)
    _check(_lib().qml_fisher(prob.ref, _ptr(F), ctypes.byref(h) if keep_plan else None,
                             _stream(prob.device)))
    return F, (Plan(h, prob) if keep_plan else None)


def cross(plan1: "Plan", plan2: "Plan", maps1=None, maps2=None):
    """Cross-QML (qml_cross): dict Wx (na x na) and, with maps, q and cl
    (na x nsims) for the columns of maps1 / maps2 filtered by each plan's C."""
    keep = []
    pr = plan1.prob
    dev = pr.device
    nsims = 0 if maps1 is None else (maps1.shape[1] if maps1.ndim == 2 else 1)
    out = {"Wx": _empty(pr.na, pr.na, dev)}
    d1 = d2 = None
    if nsims:
        d1 = _mat(maps1, pr.n, nsims, keep)
        d2 = _mat(maps2, pr.n, nsims, keep)
        out["q"] = _empty(pr.na, nsims, dev)
        out["cl"] = _empty(pr.na, nsims, dev)
    _check(_lib().qml_cross(plan1._h, plan2._h, d1, d2, nsims, _ptr(out["Wx"]),
                            _ptr(out["q"]) if nsims else None, _ptr(out["cl"]) if nsims else None,
                            _stream(dev)))
    return out


def loglike(prob: Problem, cl_theta, maps):
    """(lnL, chi2, logdet) of the columns of maps at spectra cl_theta (pix_loglike)."""
    keep = []
    nmaps = maps.shape[1] if maps.ndim == 2 else 1
    cl = _vec(cl_theta.reshape(-1) if hasattr(cl_theta, "reshape") else cl_theta, keep)
    d = _mat(maps, prob.n, nmaps, keep)
    dev = prob.device
    lnl, chi2, ld = _empty(nmaps, 1, dev), _empty(nmaps, 1, dev), _empty(1, 1, dev)
    _check(_lib().pix_loglike(prob.ref, cl, d, nmaps, _ptr(lnl), _ptr(chi2), _ptr(ld),
                              _stream(dev)))
    return lnl[:, 0], chi2[:, 0], ld[0, 0]


def loglike_batch(masks, item_mask, item_cl):
    """Batched lnL over items with mixed masks (pix_loglike_batch).

    masks: list of (Problem, maps) with maps n x nmaps; item_mask: nitems ints;
    item_cl: nitems x 6 x (lmax+1) spectra.  Returns (lnL, chi2, logdet) with
    lnL, chi2 of shape (nitems, max nmaps) and logdet (nitems,).
    """
    keep = []
    arr = (nat.LnlMask * len(masks))()
    maxmaps = 0
    for i, (prob, maps) in enumerate(masks):
        nm = maps.shape[1] if maps.ndim == 2 else 1
        arr[i].prob = prob._p
        arr[i].maps = _mat(maps, prob.n, nm, keep)
        arr[i].nmaps = nm
        maxmaps = max(maxmaps, nm)
    dev = masks[0][0].device
    nitems = len(item_mask)
    im = np.ascontiguousarray(np.asarray(item_mask), dtype=np.int32)
    keep.append(im)
    cl = _vec(item_cl.reshape(-1) if hasattr(item_cl, "reshape") else item_cl, keep)
    lnl, chi2 = _empty(maxmaps, nitems, dev), _empty(maxmaps, nitems, dev)
    ld = _empty(nitems, 1, dev)
    _check(_lib().pix_loglike_batch(arr, len(masks), nitems, im.ctypes.data, cl, maxmaps,
                                    _ptr(lnl), _ptr(chi2), _ptr(ld), _stream(dev)))
    return lnl.T, chi2.T, ld[:, 0]


def tune_set(key, value):
    """Set one entry of the library's tuning table (qml_tune_set)."""
    _check(_lib().qml_tune_set(key.encode(), int(value)))


def tune_get(key, default=None):
    """One entry of the tuning table, or `default` when absent."""
    v = ctypes.c_int64(0)
    if _lib().qml_tune_get(key.encode(), ctypes.byref(v)) != 0:
        return default
    return v.value


def tune_table():
    """The tuning table as text ("key value" per line)."""
    need = _lib().qml_tune_table(None, 0)
    buf = ctypes.create_string_buffer(int(need))
    _lib().qml_tune_table(buf, need)
    return buf.value.decode()


def tune_load(text):
    """Merge a saved tuning table (the text of tune_table) into the library's."""
    _check(_lib().qml_tune_load(text.encode()))


def autotune_batch(probs, item_mask, item_cl, streams=(4, 8, 16), graphs=(0, 1), sample=32):
    """Schedule autotuner of loglike_batch: time every (worker streams, graph
    replay) pair on the first `sample` items (CUDA events on the current
    stream, one untimed call first), store the fastest in the tuning table
    (batch_streams, batch_graphs) and return {(streams, graphs): evals/s}."""
    import torch
    item_mask = np.asarray(item_mask)[:sample]
    item_cl = item_cl[:sample]
    rates = {}
    for ns in streams:
        for gr in graphs:
            tune_set("batch_streams", ns)
            tune_set("batch_graphs", gr)
            loglike_batch(probs, item_mask, item_cl)
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record()
            loglike_batch(probs, item_mask, item_cl)
            e1.record()
            e1.synchronize()
            rates[(ns, gr)] = len(item_mask) / (e0.elapsed_time(e1) * 1e-3)
    best = max(rates, key=rates.get)
    tune_set("batch_streams", best[0])
    tune_set("batch_graphs", best[1])
    return rates


class Emulator:
    """MLP surrogate of lnL(theta) with a two-head ensemble (emu_* entry points)."""

    IN0 = 16

    def __init__(self, lo, hi, width=256, depth=4, seed=1):
        lo = np.ascontiguousarray(lo, dtype=np.float64)
        hi = np.ascontiguousarray(hi, dtype=np.float64)
        self.d, self.width, self.depth = len(lo), int(width), int(depth)
        h = ctypes.c_void_p(0)
        _check(_lib().emu_create(self.d, lo.ctypes.data, hi.ctypes.data, self.width, self.depth,
                                 int(seed), ctypes.byref(h)))
        self._h = h

    def train(self, theta, lnl, epochs=100, batch=64, lr=1e-3):
        """Train on theta (n x d) and lnl (n); returns the two heads' final MSE."""
        keep = []
        n = len(lnl)
        th = _mat(theta, n, self.d, keep)
        y = _vec(lnl, keep)
        dev = _is_torch(theta)
        fl = (ctypes.c_double * 2)()
        _check(_lib().emu_train(self._h, n, th, y, int(epochs), int(batch), float(lr),
                                ctypes.cast(fl, ctypes.c_void_p), _stream(dev)))
        return float(fl[0]), float(fl[1])

    def predict(self, theta, tol=0.05):
        """(lnL prediction, flags) for theta (n x d); tol is the accuracy target
        |dlnL| that sets the fallback threshold; flag 1 = evaluate exactly."""
        keep = []
        n = theta.shape[0]
        th = _mat(theta, n, self.d, keep)
        dev = _is_torch(theta)
        out = _empty(n, 1, dev)
        if dev:
            flags = torch.empty(n, dtype=torch.int32, device="cuda")
        else:
            flags = np.empty(n, dtype=np.int32)
        _check(_lib().emu_predict(self._h, n, th, float(tol), _ptr(out), _ptr(flags), _stream(dev)))
        return out[:, 0], flags

    def threshold(self, tol=0.05):
        """(disagreement threshold, held-out points used) for accuracy target tol."""
        thr = ctypes.c_double(0.0)
        nh = ctypes.c_int32(0)
        _check(_lib().emu_threshold(self._h, float(tol), ctypes.byref(thr), ctypes.byref(nh)))
        return thr.value, nh.value

    def params(self, head=0):
        n = _lib().emu_param_count(self._h)
        out = np.empty(n, dtype=np.float32)
        _check(_lib().emu_params(self._h, head, out.ctypes.data))
        return out

    def baseline(self):
        """(coef, sigma): the float64 baseline polynomial's coefficients (feature
        order of emu_baseline) and the residual scale of the network term."""
        coef = np.zeros(256, dtype=np.float64)
        nf = ctypes.c_int32(0)
        sig = ctypes.c_double(0.0)
        _check(_lib().emu_baseline(self._h, coef.ctypes.data, ctypes.byref(nf), ctypes.byref(sig)))
        return coef[:nf.value].copy(), sig.value

    def loss_grad(self, x, t, head=0):
        """(loss, grad) of one head on normalised inputs x (n x 16) and targets t."""
        x = np.ascontiguousarray(x, dtype=np.float64)
        t = np.ascontiguousarray(t, dtype=np.float64)
        n = _lib().emu_param_count(self._h)
        g = np.empty(n, dtype=np.float32)
        loss = ctypes.c_double(0.0)
        _check(_lib().emu_loss_grad(self._h, head, len(t), x.ctypes.data, t.ctypes.data,
                                    ctypes.byref(loss), g.ctypes.data))
        return loss.value, g

    def free(self):
        if self._h:
            _lib().emu_free(self._h)
            self._h = None

    def __del__(self):
        try:
            self.free()
        except Exception:
            pass


def potrf(A, precision=nat.QML_FP64):
    """In-place lower Cholesky of a square column-major matrix; returns ln|A|."""
    n = A.shape[0]
    dev = _is_torch(A)
    ld = _empty(1, 1, dev)
    _check(_lib().qml_potrf(n, _ptr(A), n, _ptr(ld), precision, _stream(dev)))
    return ld[0, 0]


def trsm(L, B, precision=nat.QML_FP64):
    """In-place B <- L^-1 B (both column-major)."""
    n, nrhs = B.shape
    dev = _is_torch(B)
    _check(_lib().qml_trsm(n, nrhs, _ptr(L), n, _ptr(B), n, precision, _stream(dev)))
    return B


def gemm(A, B, C=None, transA=False, transB=False, alpha=1.0, beta=0.0, lower=False,
         precision=nat.QML_FP64):
    """C <- alpha op(A) op(B) + beta C (column-major operands)."""
    m = A.shape[1] if transA else A.shape[0]
    kk = A.shape[0] if transA else A.shape[1]
    nn = B.shape[0] if transB else B.shape[1]
    dev = _is_torch(A)
    if C is None:
        C = _empty(m, nn, dev)
        if dev:
            C.zero_()
        else:
            C[:] = 0.0
    _check(_lib().qml_gemm(int(transA), int(transB), m, nn, kk, alpha, _ptr(A), max(1, A.shape[0]),
                           _ptr(B), max(1, B.shape[0]), beta, _ptr(C), max(1, C.shape[0]), int(lower),
                           precision, _stream(dev)))
    return C
