"""Thin ctypes binding of librsx (include/rsx.h): argument marshalling only.

Every computation runs in the CUDA library.  Tensors are PyTorch CUDA tensors used as
device memory; the stream is torch's current stream unless one is given.  If the
library has not been built the first call raises: there is no CPU fallback.
"""
import ctypes
import os

import torch

_HERE = os.path.dirname(os.path.abspath(__file__))
# RSX_CHECKED=1 selects the bounds-checked build (librsx_checked.so, built by
# build(checked=True)): same ABI, the FFT passes report out-of-range indices as RSX_EBOUNDS
LIB_PATH = os.path.join(_HERE, "librsx_checked.so" if os.environ.get("RSX_CHECKED") == "1" else "librsx.so")

RSX_OK, RSX_EINVAL, RSX_ENOMEM, RSX_ECUDA, RSX_ENOTPD, RSX_ETIMEOUT, RSX_EUNSUPPORTED, RSX_EBOUNDS = range(8)
RSX_FP64, RSX_FP32 = 0, 1
RSX_FAULT_NONE, RSX_FAULT_ALLOC, RSX_FAULT_PIVOT = 0, 1, 2
ERROR_NAMES = {1: "RSX_EINVAL", 2: "RSX_ENOMEM", 3: "RSX_ECUDA", 4: "RSX_ENOTPD", 5: "RSX_ETIMEOUT",
               6: "RSX_EUNSUPPORTED", 7: "RSX_EBOUNDS"}

# exported symbol -> ctypes argument types (mirrors include/rsx.h)
_P = ctypes.c_void_p
_I = ctypes.c_int
_D = ctypes.c_double
SIGNATURES = {
    "rsx_create": [ctypes.POINTER(_P), _I, _I, _I, _D, _I, _I],
    "rsx_destroy": [_P],
    "rsx_last_error": [_P],
    "rsx_set_workspace_limit": [_P, ctypes.c_size_t],
    "rsx_build_pair_densities": [_P, _P, _I, _P, _I, _P, _P],
    "rsx_exchange_apply": [_P, _P, _I, _P, _I, _P, _P],
    "rsx_exchange_apply_noalloc": [_P, _P, _I, _P, _I, _P, _P],
    "rsx_poisson": [_P, _P, _P, _P],
    "rsx_ace_build": [_P, _P, _I, _P, _P, _P],
    "rsx_ace_apply": [_P, _P, _I, _P, _I, _P, _P],
    "rsx_gram": [_P, _P, _I, _P, _I, _P, _P],
    "rsx_ace_factor": [_P, _P, _P, _I, _P, _P],
    "rsx_casida_K": [_P, _P, _I, _P, _I, _P, _P],
    "rsx_casida_Kd": [_P, _P, _I, _P, _I, _P, _P],
    "rsx_casida_K_uhf": [_P, _P, _I, _P, _I, _P, _I, _P, _I, _P, _P],
    "rsx_casida_solve_uhf": [_P, _P, _I, _P, _I, _P, _I, _P, _I, _P, _P, _P, _I, _P, _P, _P],
    "rsx_casida_solve": [_P, _P, _I, _P, _I, _P, _P, _D, _I, _P, _P, _P],
    "rsx_casida_solve_full": [_P, _P, _I, _P, _I, _P, _P, _D, _I, _P, _P, _P],
    "rsx_casida_dipoles": [_P, _P, _I, _P, _I, _P, _P],
    "rsx_casida_oscillator": [_P, _P, _P, _I, _I, _P, _P, _P],
    "rsx_strength_function": [_P, _P, _P, _I, _D, _P, _I, _P, _P],
    "rsx_syrk_bf16x3": [_P, _P, _P, _I, ctypes.c_longlong, _P, _P],
    "rsx_eig_create": [ctypes.POINTER(_P), _I, _D, _P, ctypes.c_float, _I, _I],
    "rsx_eig_init": [_P, _P, _P],
    "rsx_eig_step": [_P, _P, _I, ctypes.POINTER(_D), _P],
    "rsx_eig_orbitals": [_P, _P, _P],
    "rsx_eig_residual": [_P, _P, _P],
    "rsx_eig_last_error": [_P],
    "rsx_eig_energy64": [_P, ctypes.POINTER(_D), _P],
    "rsx_eig_destroy": [_P],
    "rsx_eig_set_exchange": [_P, _P, _P, _I, _I],
    "rsx_eig_set_mask": [_P, _P],
    "rsx_eig_refresh": [_P, ctypes.POINTER(_D), _P],
    "rsx_scf_create": [ctypes.POINTER(_P), _P, _P, _I, _I, ctypes.c_float],
    "rsx_scf_init": [_P, _P, _P],
    "rsx_scf_step": [_P, _I, ctypes.POINTER(_D), _P],
    "rsx_scf_set_mixing": [_P, _I],
    "rsx_scf_set_mask": [_P, _P],
    "rsx_scf_orbitals": [_P, _P, _P],
    "rsx_scf_last_error": [_P],
    "rsx_scf_destroy": [_P],
    "rsx_net_create": [ctypes.POINTER(_P), _I],
    "rsx_net_param_count": [],
    "rsx_net_set_params": [_P, ctypes.POINTER(ctypes.c_float), _I],
    "rsx_net_get_params": [_P, ctypes.POINTER(ctypes.c_float), _I],
    "rsx_net_forward": [_P, _P, _I, _I, _I, _I, _P, _P],
    "rsx_net_loss_grad": [_P, _P, _P, _I, _I, _I, _I, _I, ctypes.POINTER(_D), ctypes.POINTER(ctypes.c_float), _P],
    "rsx_net_train_step": [_P, _P, _P, _I, _I, _I, _I, _I, ctypes.c_float, ctypes.POINTER(_D), _P],
    "rsx_net_sync_status": [_P, _P],
    "rsx_net_last_error": [_P],
    "rsx_net_destroy": [_P],
    "rsx_batch_create": [ctypes.POINTER(_P), _I, ctypes.POINTER(_I), ctypes.POINTER(_I), _D, _I],
    "rsx_batch_bind": [_P, ctypes.POINTER(_P), ctypes.POINTER(_P), ctypes.POINTER(_P)],
    "rsx_batch_run": [_P, _P],
    "rsx_batch_sync_status": [_P, _P],
    "rsx_batch_last_error": [_P],
    "rsx_batch_destroy": [_P],
    "rsx_autotune": [_P, _I, _I, ctypes.c_char_p, ctypes.POINTER(_I), ctypes.POINTER(_I), ctypes.POINTER(_D)],
    "rsx_set_tuning": [_P, _I, _I],
    "rsx_get_tuning": [_P, _P],
    "rsx_set_tuning_ex": [_P, _P],
    "rsx_autotune_ex": [_P, _I, _I, ctypes.c_char_p, _P, ctypes.POINTER(_D)],
    "rsx_sync_status": [_P, _P],
    "rsx_set_wait_limit": [_P, ctypes.c_longlong],
    "rsx_inject_fault": [_P, _I, _I],
    "rsx_profile_enable": [_P, _I],
    "rsx_profile_reset": [_P],
    "rsx_profile_read": [_P, _I, ctypes.POINTER(_D), ctypes.POINTER(ctypes.c_longlong)],
    "rsx_kernel_count": [],
    "rsx_kernel_name": [_I],
}

_lib = None


class Tuning(ctypes.Structure):
    """rsx_tuning: knobs of the pair-solve path (performance only)."""
    _fields_ = [("p2_threads", _I), ("chunk_outputs", _I), ("p1_group", _I), ("p2_global", _I), ("p2_lanes", _I)]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_}


class RsxError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__(f"{ERROR_NAMES.get(code, code)}: {msg}")
        self.code = code


def load(path=LIB_PATH):
    """Open librsx.so once and declare its signatures."""
    global _lib
    if _lib is None:
        if not os.path.exists(path):
            raise RuntimeError(f"librsx.so not found at {path}: build it with __graft_entry__.build()")
        lib = ctypes.CDLL(path)
        for name, args in SIGNATURES.items():
            f = getattr(lib, name)
            f.argtypes = args
            f.restype = (ctypes.c_char_p if name in ("rsx_last_error", "rsx_kernel_name", "rsx_batch_last_error",
                                                     "rsx_eig_last_error", "rsx_net_last_error",
                                                     "rsx_scf_last_error")
                         else ctypes.c_int)
        _lib = lib
    return _lib


def _ptr(t):
    return ctypes.c_void_p(t.data_ptr()) if t is not None else ctypes.c_void_p(0)


def _stream(stream):
    s = stream if stream is not None else torch.cuda.current_stream()
    return ctypes.c_void_p(s.cuda_stream)


class Context:
    """One rsx context: box (nz, ny, nx), spacing h, precision 'fp32' or 'fp64'."""

    def __init__(self, shape, h, precision="fp32", device=0):
        self.lib = load()
        self.shape = tuple(int(s) for s in shape)
        self.h = float(h)
        self.precision = precision
        self.dtype = torch.float32 if precision == "fp32" else torch.float64
        self.device = torch.device("cuda", device)
        self.N = self.shape[0] * self.shape[1] * self.shape[2]
        h_ = ctypes.c_void_p()
        code = self.lib.rsx_create(ctypes.byref(h_), self.shape[0], self.shape[1], self.shape[2], self.h,
                                   RSX_FP32 if precision == "fp32" else RSX_FP64, device)
        if code != RSX_OK:
            raise RsxError(code, "rsx_create failed")
        self.handle = h_

    def close(self):
        if getattr(self, "handle", None):
            self.lib.rsx_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def _check(self, code):
        if code != RSX_OK:
            raise RsxError(code, self.lib.rsx_last_error(self.handle).decode())

    def _orb(self, t, name):
        if not (t.is_cuda and t.dtype == self.dtype and t.is_contiguous()):
            raise ValueError(f"{name}: need a contiguous {self.dtype} CUDA tensor")
        if t.numel() % self.N:
            raise ValueError(f"{name}: size is not a multiple of the grid")
        return t.numel() // self.N

    def _new(self, n):
        return torch.empty((n,) + self.shape, dtype=self.dtype, device=self.device)

    def set_workspace_limit(self, nbytes):
        self._check(self.lib.rsx_set_workspace_limit(self.handle, int(nbytes)))

    def autotune(self, nocc, npsi, cache=None):
        """Time the exchange-path candidates on the device and apply the fastest."""
        t, ms = Tuning(), ctypes.c_double()
        self._check(self.lib.rsx_autotune_ex(self.handle, int(nocc), int(npsi),
                                             cache.encode() if cache else None,
                                             ctypes.byref(t), ctypes.byref(ms)))
        return dict(t.as_dict(), best_ms=ms.value)

    def get_tuning(self):
        t = Tuning()
        self._check(self.lib.rsx_get_tuning(self.handle, ctypes.byref(t)))
        return t.as_dict()

    def set_tuning(self, p2_threads=None, chunk_outputs=None, p1_group=None, p2_global=None, p2_lanes=None):
        """Set any of the knobs (the others keep their values)."""
        t = Tuning()
        self._check(self.lib.rsx_get_tuning(self.handle, ctypes.byref(t)))
        for k, v in (("p2_threads", p2_threads), ("chunk_outputs", chunk_outputs), ("p1_group", p1_group),
                     ("p2_global", p2_global), ("p2_lanes", p2_lanes)):
            if v is not None:
                setattr(t, k, int(v))
        self._check(self.lib.rsx_set_tuning_ex(self.handle, ctypes.byref(t)))

    def pair_densities(self, a, b, out=None, stream=None):
        na, nb = self._orb(a, "a"), self._orb(b, "b")
        out = self._new(na * nb) if out is None else out
        self._check(self.lib.rsx_build_pair_densities(self.handle, _ptr(a), na, _ptr(b), nb, _ptr(out),
                                                      _stream(stream)))
        return out

    def exchange_apply(self, phi, psi, out=None, stream=None):
        nocc, npsi = self._orb(phi, "phi"), self._orb(psi, "psi")
        out = self._new(npsi) if out is None else out
        self._check(self.lib.rsx_exchange_apply(self.handle, _ptr(phi), nocc, _ptr(psi), npsi, _ptr(out),
                                                _stream(stream)))
        return out

    def exchange_apply_noalloc(self, phi, psi, out, stream=None):
        """Same as exchange_apply, but the library allocates nothing (fixed 64 MiB scratch)."""
        nocc, npsi = self._orb(phi, "phi"), self._orb(psi, "psi")
        self._check(self.lib.rsx_exchange_apply_noalloc(self.handle, _ptr(phi), nocc, _ptr(psi), npsi, _ptr(out),
                                                        _stream(stream)))
        return out

    def poisson(self, rho, V=None, stream=None):
        """Isolated-boundary potential of one density (the solve behind Eq. 2)."""
        if self._orb(rho, "rho") != 1:
            raise ValueError("rho: one density")
        V = torch.empty_like(rho) if V is None else V
        self._check(self.lib.rsx_poisson(self.handle, _ptr(rho), _ptr(V), _stream(stream)))
        return V

    def ace_build(self, phi, xi=None, M=None, stream=None):
        nocc = self._orb(phi, "phi")
        xi = self._new(nocc) if xi is None else xi
        self._check(self.lib.rsx_ace_build(self.handle, _ptr(phi), nocc, _ptr(xi), _ptr(M), _stream(stream)))
        return xi

    def gram(self, a, b, C=None, stream=None):
        """C[i][j] = h^3 <a_i, b_j> (FP64)."""
        na, nb = self._orb(a, "a"), self._orb(b, "b")
        C = torch.empty((na, nb), dtype=torch.float64, device=self.device) if C is None else C
        self._check(self.lib.rsx_gram(self.handle, _ptr(a), na, _ptr(b), nb, _ptr(C), _stream(stream)))
        return C

    def ace_factor(self, M, W, xi=None, stream=None):
        """Symmetrise M in place, -M = L L^T (FP64), xi = L^-1 W (Eqs. 11-12 after W)."""
        nocc = self._orb(W, "W")
        xi = self._new(nocc) if xi is None else xi
        self._check(self.lib.rsx_ace_factor(self.handle, _ptr(M), _ptr(W), nocc, _ptr(xi), _stream(stream)))
        return xi

    def ace_apply(self, xi, psi, out=None, stream=None):
        nxi, npsi = self._orb(xi, "xi"), self._orb(psi, "psi")
        out = self._new(npsi) if out is None else out
        self._check(self.lib.rsx_ace_apply(self.handle, _ptr(xi), nxi, _ptr(psi), npsi, _ptr(out),
                                           _stream(stream)))
        return out

    def casida_K(self, phi_occ, phi_virt, K=None, stream=None):
        no, nv = self._orb(phi_occ, "phi_occ"), self._orb(phi_virt, "phi_virt")
        nt = no * nv
        K = torch.empty((nt, nt), dtype=torch.float64, device=self.device) if K is None else K
        self._check(self.lib.rsx_casida_K(self.handle, _ptr(phi_occ), no, _ptr(phi_virt), nv, _ptr(K),
                                          _stream(stream)))
        return K

    def casida_Kd(self, phi_occ, phi_virt, Kd=None, stream=None):
        no, nv = self._orb(phi_occ, "phi_occ"), self._orb(phi_virt, "phi_virt")
        nt = no * nv
        Kd = torch.empty((nt, nt), dtype=torch.float64, device=self.device) if Kd is None else Kd
        self._check(self.lib.rsx_casida_Kd(self.handle, _ptr(phi_occ), no, _ptr(phi_virt), nv, _ptr(Kd),
                                           _stream(stream)))
        return Kd

    def casida_K_uhf(self, occ_a, virt_a, occ_b=None, virt_b=None, K=None, stream=None):
        """(ia|jb) over alpha then beta transitions (spin-orbital form, Eqs. 4-5)."""
        noa, nva = self._orb(occ_a, "occ_a"), self._orb(virt_a, "virt_a")
        nob = self._orb(occ_b, "occ_b") if occ_b is not None else 0
        nvb = self._orb(virt_b, "virt_b") if virt_b is not None else 0
        nt = noa * nva + (nob * nvb if nob and nvb else 0)
        K = torch.empty((nt, nt), dtype=torch.float64, device=self.device) if K is None else K
        self._check(self.lib.rsx_casida_K_uhf(self.handle, _ptr(occ_a), noa, _ptr(virt_a), nva, _ptr(occ_b), nob,
                                              _ptr(virt_b), nvb, _ptr(K), _stream(stream)))
        return K

    def casida_solve_uhf(self, eo_a, ev_a, eo_b, ev_b, K, Kd_a=None, Kd_b=None, nroots=10, vectors=False,
                         stream=None):
        """Lowest roots of diag + K - blockdiag(Kd_a, Kd_b); eps as device float64 tensors."""
        nb_t = eo_b.numel() * ev_b.numel() if eo_b is not None and ev_b is not None else 0
        nt = eo_a.numel() * ev_a.numel() + nb_t
        omega = torch.empty(nroots, dtype=torch.float64, device=self.device)
        X = torch.empty((nroots, nt), dtype=torch.float64, device=self.device) if vectors else None
        self._check(self.lib.rsx_casida_solve_uhf(
            self.handle, _ptr(eo_a), eo_a.numel(), _ptr(ev_a), ev_a.numel(), _ptr(eo_b),
            eo_b.numel() if eo_b is not None else 0, _ptr(ev_b), ev_b.numel() if ev_b is not None else 0,
            _ptr(K), _ptr(Kd_a), _ptr(Kd_b), int(nroots), _ptr(omega), _ptr(X), _stream(stream)))
        return (omega, X) if vectors else omega

    def casida_solve(self, eps_occ, eps_virt, K, Kd=None, delta_M=2.0, nroots=10, vectors=False, stream=None):
        no, nv = eps_occ.numel(), eps_virt.numel()
        nt = no * nv
        omega = torch.empty(nroots, dtype=torch.float64, device=self.device)
        X = torch.empty((nroots, nt), dtype=torch.float64, device=self.device) if vectors else None
        self._check(self.lib.rsx_casida_solve(self.handle, _ptr(eps_occ), no, _ptr(eps_virt), nv, _ptr(K),
                                              _ptr(Kd), float(delta_M), int(nroots), _ptr(omega), _ptr(X),
                                              _stream(stream)))
        return (omega, X) if vectors else omega

    def casida_solve_full(self, eps_occ, eps_virt, K, Kd=None, delta_M=2.0, nroots=10, vectors=False, stream=None):
        """Full TDHF (A and B) in the half-size form: omega and, with vectors, X + Y."""
        no, nv = eps_occ.numel(), eps_virt.numel()
        nt = no * nv
        omega = torch.empty(nroots, dtype=torch.float64, device=self.device)
        XpY = torch.empty((nroots, nt), dtype=torch.float64, device=self.device) if vectors else None
        self._check(self.lib.rsx_casida_solve_full(self.handle, _ptr(eps_occ), no, _ptr(eps_virt), nv, _ptr(K),
                                                   _ptr(Kd), float(delta_M), int(nroots), _ptr(omega), _ptr(XpY),
                                                   _stream(stream)))
        return (omega, XpY) if vectors else omega

    def casida_dipoles(self, phi_occ, phi_virt, stream=None):
        """<i|r_d|a> as a [3][nocc * nvirt] FP64 tensor (x, y, z)."""
        no, nv = self._orb(phi_occ, "phi_occ"), self._orb(phi_virt, "phi_virt")
        dip = torch.empty((3, no * nv), dtype=torch.float64, device=self.device)
        self._check(self.lib.rsx_casida_dipoles(self.handle, _ptr(phi_occ), no, _ptr(phi_virt), nv, _ptr(dip),
                                                _stream(stream)))
        return dip

    def oscillator_strengths(self, omega, X, dip, stream=None):
        nroots, nt = X.shape
        f = torch.empty(nroots, dtype=torch.float64, device=self.device)
        self._check(self.lib.rsx_casida_oscillator(self.handle, _ptr(omega), _ptr(X), nroots, nt, _ptr(dip), _ptr(f),
                                                   _stream(stream)))
        return f

    def strength_function(self, omega, f, gamma, grid, stream=None):
        S = torch.empty(grid.numel(), dtype=torch.float64, device=self.device)
        self._check(self.lib.rsx_strength_function(self.handle, _ptr(omega), _ptr(f), omega.numel(), float(gamma),
                                                   _ptr(grid), grid.numel(), _ptr(S), _stream(stream)))
        return S

    def syrk_bf16x3(self, hi, lo, C=None, stream=None):
        """C = H H^T + H L^T + L H^T for bf16 panels [n][ld] (n % 128 == 0, ld % 64 == 0)."""
        n, ld = hi.shape
        C = torch.empty((n, n), dtype=torch.float64, device=self.device) if C is None else C
        self._check(self.lib.rsx_syrk_bf16x3(self.handle, _ptr(hi), _ptr(lo), n, ld, _ptr(C), _stream(stream)))
        return C

    def profile(self, on=True):
        self._check(self.lib.rsx_profile_enable(self.handle, 1 if on else 0))

    def profile_reset(self):
        self._check(self.lib.rsx_profile_reset(self.handle))

    def profile_read(self):
        """{kernel name: (total ms, launches)} for every kernel launched since the last reset."""
        out = {}
        for k in range(self.lib.rsx_kernel_count()):
            ms, n = ctypes.c_double(), ctypes.c_longlong()
            self._check(self.lib.rsx_profile_read(self.handle, k, ctypes.byref(ms), ctypes.byref(n)))
            if n.value:
                out[self.lib.rsx_kernel_name(k).decode()] = (ms.value, n.value)
        return out

    def sync(self, stream=None):
        self._check(self.lib.rsx_sync_status(self.handle, _stream(stream)))

    def set_wait_limit(self, spins):
        """Spin rounds of the bounded grid waits (testing aid; < 0 restores the default)."""
        self._check(self.lib.rsx_set_wait_limit(self.handle, int(spins)))

    def inject_fault(self, kind, after=0):
        """Host-side fault injection (testing aid): RSX_FAULT_ALLOC, RSX_FAULT_PIVOT, RSX_FAULT_NONE."""
        self._check(self.lib.rsx_inject_fault(self.handle, int(kind), int(after)))


class Batch:
    """Uneven batch of molecules: W_m = Vx[phi_m] phi_m and ACE projectors xi_m for all m,
    in persistent launches replayed from a captured CUDA graph (FP32)."""

    def __init__(self, edges, nocc, h, device=0):
        self.lib = load()
        self.edges = [int(e) for e in edges]
        self.nocc = [int(k) for k in nocc]
        self.nmol = len(self.edges)
        self.device = torch.device("cuda", device)
        h_ = ctypes.c_void_p()
        E = (ctypes.c_int * self.nmol)(*self.edges)
        K = (ctypes.c_int * self.nmol)(*self.nocc)
        code = self.lib.rsx_batch_create(ctypes.byref(h_), self.nmol, E, K, float(h), device)
        if code != RSX_OK:
            raise RsxError(code, "rsx_batch_create failed")
        self.handle = h_
        self._bound = None

    def _check(self, code):
        if code != RSX_OK:
            raise RsxError(code, self.lib.rsx_batch_last_error(self.handle).decode())

    def bind(self, phi, W, xi):
        """phi, W, xi: lists of contiguous float32 CUDA tensors [nocc_m, e, e, e]."""
        for m in range(self.nmol):
            shape = (self.nocc[m],) + (self.edges[m],) * 3
            for t in (phi[m], W[m], xi[m]):
                if not (t.is_cuda and t.dtype == torch.float32 and t.is_contiguous() and tuple(t.shape) == shape):
                    raise ValueError(f"molecule {m}: need contiguous float32 CUDA tensors of shape {shape}")
        arr = lambda ts: (ctypes.c_void_p * self.nmol)(*[t.data_ptr() for t in ts])
        self._check(self.lib.rsx_batch_bind(self.handle, arr(phi), arr(W), arr(xi)))
        self._bound = (phi, W, xi)

    def run(self, stream=None):
        self._check(self.lib.rsx_batch_run(self.handle, _stream(stream)))

    def sync(self, stream=None):
        self._check(self.lib.rsx_batch_sync_status(self.handle, _stream(stream)))

    def close(self):
        if getattr(self, "handle", None):
            self.lib.rsx_batch_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class Net:
    """The learned preconditioner network (3 conv3d layers, bf16 weights, FP32 accumulation)."""

    def __init__(self, params=None, device=0):
        import numpy as np
        self.lib = load()
        self.device = torch.device("cuda", device)
        h_ = ctypes.c_void_p()
        code = self.lib.rsx_net_create(ctypes.byref(h_), device)
        if code != RSX_OK:
            raise RsxError(code, "rsx_net_create failed")
        self.handle = h_
        self.nparams = self.lib.rsx_net_param_count()
        if params is not None:
            self.set_params(params)

    def _check(self, code):
        if code != RSX_OK:
            raise RsxError(code, self.lib.rsx_net_last_error(self.handle).decode())

    def set_params(self, params):
        import numpy as np
        p = np.ascontiguousarray(params, dtype=np.float32)
        self._check(self.lib.rsx_net_set_params(self.handle, p.ctypes.data_as(ctypes.POINTER(ctypes.c_float)), p.size))

    def get_params(self):
        import numpy as np
        p = np.empty(self.nparams, dtype=np.float32)
        self._check(self.lib.rsx_net_get_params(self.handle, p.ctypes.data_as(ctypes.POINTER(ctypes.c_float)), p.size))
        return p

    def forward(self, x, out=None, stream=None):
        B, C, D, H, W = x.shape
        out = torch.empty((B, D, H, W), dtype=torch.float32, device=self.device) if out is None else out
        self._check(self.lib.rsx_net_forward(self.handle, _ptr(x), B, D, H, W, _ptr(out), _stream(stream)))
        return out

    def loss_grad(self, x, target, border=0, stream=None):
        import numpy as np
        B, C, D, H, W = x.shape
        loss = ctypes.c_double()
        g = np.empty(self.nparams, dtype=np.float32)
        self._check(self.lib.rsx_net_loss_grad(self.handle, _ptr(x), _ptr(target), B, D, H, W, int(border),
                                               ctypes.byref(loss), g.ctypes.data_as(ctypes.POINTER(ctypes.c_float)),
                                               _stream(stream)))
        return loss.value, g

    def train_step(self, x, target, lr, border=0, stream=None):
        B, C, D, H, W = x.shape
        loss = ctypes.c_double()
        self._check(self.lib.rsx_net_train_step(self.handle, _ptr(x), _ptr(target), B, D, H, W, int(border),
                                                float(lr), ctypes.byref(loss), _stream(stream)))
        return loss.value

    def sync(self, stream=None):
        """Wait for the network's kernels on the stream; raise on a deferred device error."""
        self._check(self.lib.rsx_net_sync_status(self.handle, _stream(stream)))

    def close(self):
        if getattr(self, "handle", None):
            self.lib.rsx_net_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class Eigensolver:
    """Block preconditioned eigensolver for H = -1/2 Lap + V on an n^3 box (FP32)."""

    def __init__(self, V, h, nband, vscale=1.0, device=0):
        self.lib = load()
        self.V = V
        self.n = V.shape[0]
        self.nband = nband
        h_ = ctypes.c_void_p()
        code = self.lib.rsx_eig_create(ctypes.byref(h_), self.n, float(h), _ptr(V), float(vscale), nband, device)
        if code != RSX_OK:
            raise RsxError(code, "rsx_eig_create failed")
        self.handle = h_

    def _check(self, code):
        if code != RSX_OK:
            raise RsxError(code, self.lib.rsx_eig_last_error(self.handle).decode())

    def init(self, psi0, stream=None):
        self._check(self.lib.rsx_eig_init(self.handle, _ptr(psi0), _stream(stream)))

    def step(self, net=None, sweeps=3, stream=None):
        th = (ctypes.c_double * self.nband)()
        self._check(self.lib.rsx_eig_step(self.handle, net.handle if net is not None else None, int(sweeps), th,
                                          _stream(stream)))
        return list(th)

    def energy64(self, stream=None):
        """FP64 Rayleigh-Ritz energy trace(S^-1 <Psi, H Psi>) of the current orbitals."""
        e = ctypes.c_double()
        self._check(self.lib.rsx_eig_energy64(self.handle, ctypes.byref(e), _stream(stream)))
        return e.value

    def set_exchange(self, src=None, mode=0, ctx=None):
        """Exchange term of H: mode 0 none, 1 ACE with projectors src, 2 exact Vx[src] via ctx."""
        self._xsrc = src                      # the library keeps the pointer
        count = src.shape[0] if src is not None else 0
        self._check(self.lib.rsx_eig_set_exchange(self.handle, ctx.handle if ctx is not None else None,
                                                  _ptr(src), int(count), int(mode)))

    def set_mask(self, mask=None):
        """Spherical domain: H restricted to mask == 1 (device float32 [n, n, n]); None clears."""
        self._mask = mask                     # the library keeps the pointer
        self._check(self.lib.rsx_eig_set_mask(self.handle, _ptr(mask)))

    def refresh(self, stream=None):
        th = (ctypes.c_double * self.nband)()
        self._check(self.lib.rsx_eig_refresh(self.handle, th, _stream(stream)))
        return list(th)

    def orbitals(self, out=None, stream=None):
        out = torch.empty((self.nband,) + tuple(self.V.shape), dtype=torch.float32, device=self.V.device) \
            if out is None else out
        self._check(self.lib.rsx_eig_orbitals(self.handle, _ptr(out), _stream(stream)))
        return out

    def residual(self, out=None, stream=None):
        out = torch.empty((self.nband,) + tuple(self.V.shape), dtype=torch.float32, device=self.V.device) \
            if out is None else out
        self._check(self.lib.rsx_eig_residual(self.handle, _ptr(out), _stream(stream)))
        return out

    def close(self):
        if getattr(self, "handle", None):
            self.lib.rsx_eig_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class SCF:
    """Closed-shell Hartree-Fock SCF with ACE or exact exchange (Sec. 3.1-3.2) on the
    cubic box of an FP32 Context; V_ext a device [n, n, n] float32 tensor."""

    FIELDS = ("energy", "one_body", "hartree", "exchange", "reldens", "theta_sum")

    def __init__(self, ctx, v_ext, nocc, ace=True, alpha=0.3, mix="density", mask=None):
        self.lib = load()
        self.ctx = ctx                        # kept alive: the library holds both pointers
        self.v_ext = v_ext
        self.nocc = nocc
        h_ = ctypes.c_void_p()
        code = self.lib.rsx_scf_create(ctypes.byref(h_), ctx.handle, _ptr(v_ext), int(nocc), int(bool(ace)),
                                       float(alpha))
        if code != RSX_OK:
            raise RsxError(code, "rsx_scf_create failed")
        self.handle = h_
        self.mix = mix
        self.mask = mask                      # the library keeps the pointer
        if mask is not None:
            self._check(self.lib.rsx_scf_set_mask(self.handle, _ptr(mask)))

    def _check(self, code):
        if code != RSX_OK:
            raise RsxError(code, self.lib.rsx_scf_last_error(self.handle).decode())

    def init(self, psi0, stream=None):
        """Start from psi0; `mix` ('density' or 'states') applies from here."""
        if self.mix not in ("density", "states"):
            raise ValueError("mix: 'density' or 'states'")
        self._check(self.lib.rsx_scf_init(self.handle, _ptr(psi0), _stream(stream)))
        self._check(self.lib.rsx_scf_set_mixing(self.handle, int(self.mix == "states")))

    def step(self, inner=2, stream=None):
        """One SCF iteration; returns a dict of the six reported quantities."""
        out = (ctypes.c_double * 6)()
        self._check(self.lib.rsx_scf_step(self.handle, int(inner), out, _stream(stream)))
        return dict(zip(self.FIELDS, list(out)))

    def orbitals(self, out=None, stream=None):
        out = torch.empty((self.nocc,) + tuple(self.v_ext.shape), dtype=torch.float32, device=self.v_ext.device) \
            if out is None else out
        self._check(self.lib.rsx_scf_orbitals(self.handle, _ptr(out), _stream(stream)))
        return out

    def close(self):
        if getattr(self, "handle", None):
            self.lib.rsx_scf_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
