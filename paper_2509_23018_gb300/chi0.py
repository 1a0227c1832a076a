"""Python binding of the chi0 C ABI (argument marshalling only).

Names follow include/gw_chi0.h: ``create``, ``set_bands``, ``set_gsphere``,
``compute``, ``compute_batch``, ``pair_elements``, ``contract``, ``adjoint``,
``subspace_basis``, ``compute_subspace``, ``epsilon_inverse``, ``compute_real``,
``jvp``, ``sigma_gpp``, ``keep_pair_elements``, ``streams``, ``sync``, ``destroy``.
Torch supplies device memory and the stream; every arithmetic step runs in the
CUDA library.  Complex tensors are complex128 (interleaved re/im doubles).

Typical use (one q-point)::

    h = Chi0((48, 48, 48), prec="ozaki", nslices=7, mtxel="twofloat")
    h.set_bands(0, 0, gvec_psi, c_valence, e_valence)     # kind 0: valence at k+q
    h.set_bands(0, 1, gvec_psi, c_conduction, e_conduction)
    h.set_gsphere(0, gvec_chi)
    (chi,) = h.compute(0, [0.0, 2.0])                    # [n_omega, N_G, N_G]
"""
from __future__ import annotations

import ctypes
from typing import Sequence

import torch

from . import _lib


class GwError(RuntimeError):
    def __init__(self, status: int, msg: str):
        super().__init__(f"{_lib.STATUS_NAMES.get(status, status)}: {msg}")
        self.status = status


def _ptr(t):
    return ctypes.c_void_p(t.data_ptr()) if t is not None else ctypes.c_void_p(0)


def _stream_handle():
    return ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)


PREC = {"fp64": _lib.GW_PREC_FP64, "ozaki": _lib.GW_PREC_OZAKI_BF16, "ozaki_bf16": _lib.GW_PREC_OZAKI_BF16}
MTXEL = {"fp64": _lib.GW_MTXEL_FP64, "twofloat": _lib.GW_MTXEL_TWOFLOAT}


class Chi0:
    """One handle of the library (one device, one stream at a time)."""

    def __init__(self, grid: Sequence[int], nq: int = 1, prec: str = "fp64", nslices: int = 6,
                 pair_chunk: int = 8192, mem_budget_bytes: int = 0, device: int | None = None,
                 mtxel: str = "fp64", single_stream: bool = False):
        self.lib = _lib.load()
        dev = torch.cuda.current_device() if device is None else device
        d = _lib.Desc()
        for a in range(3):
            d.n[a] = int(grid[a])
        d.nq, d.prec, d.nslices = int(nq), PREC[prec], int(nslices)
        d.pair_chunk, d.mem_budget_bytes, d.device = int(pair_chunk), int(mem_budget_bytes), int(dev)
        d.mtxel_prec = MTXEL[mtxel]
        d.single_stream = 1 if single_stream else 0
        h = ctypes.c_void_p()
        with torch.cuda.device(dev):
            st = self.lib.gw_chi0_create(ctypes.byref(h), ctypes.byref(d), _stream_handle())
        if st != 0:
            raise GwError(st, "gw_chi0_create failed")
        self.h = h
        self.grid = tuple(int(x) for x in grid)
        self.nq, self.prec, self.device = int(nq), prec, dev
        self.ng = {}
        self.nb = {}
        self.ngpsi = {}

    # -------------------------------------------------------------- helpers
    def _check(self, st):
        if st != 0:
            raise GwError(st, self.lib.gw_chi0_last_error(self.h).decode())

    def _use_current_stream(self):
        self._check(self.lib.gw_chi0_set_stream(self.h, _stream_handle()))

    # -------------------------------------------------------------- ABI calls
    def set_bands(self, iq: int, kind: int, gvec: torch.Tensor, coeff: torch.Tensor, energy: torch.Tensor):
        gvec = gvec.to(device=f"cuda:{self.device}", dtype=torch.int32).contiguous()
        coeff = coeff.to(device=f"cuda:{self.device}", dtype=torch.complex128).contiguous()
        energy = energy.to(device=f"cuda:{self.device}", dtype=torch.float64).contiguous()
        self._use_current_stream()
        self._check(self.lib.gw_chi0_set_bands(self.h, int(iq), int(kind), coeff.shape[0], coeff.shape[1],
                                               _ptr(gvec), _ptr(coeff), _ptr(energy)))
        key = ("c",) if kind == 1 else ("v", iq)
        self.nb[key] = coeff.shape[0]
        self.ngpsi[key] = coeff.shape[1]

    def set_gsphere(self, iq: int, gvec: torch.Tensor):
        gvec = gvec.to(device=f"cuda:{self.device}", dtype=torch.int32).contiguous()
        self._use_current_stream()
        self._check(self.lib.gw_chi0_set_gsphere(self.h, int(iq), gvec.shape[0], _ptr(gvec)))
        self.ng[iq] = gvec.shape[0]

    def compute_batch(self, iq: Sequence[int], omega: Sequence[float], out: torch.Tensor | None = None,
                      diag: bool = False):
        """Batched chi0 (all slots and frequencies, graph-captured); same packing as ``compute``."""
        return self.compute(iq, omega, out=out, diag=diag, _batch=True)

    def tuning(self):
        a, b, c = ctypes.c_int(), ctypes.c_int(), ctypes.c_int()
        n = self.lib.gw_chi0_tuning(self.h, ctypes.byref(a), ctypes.byref(b), ctypes.byref(c))
        return {"tile_f64": a.value, "waves_f64": b.value, "tile_split": c.value, "shapes_tuned": n}

    def compute(self, iq: Sequence[int] | int, omega: Sequence[float], out: torch.Tensor | None = None,
                diag: bool = False, _batch: bool = False):
        """chi0 blocks: list (per slot) of [nw, ng, ng] complex128 views into one packed buffer."""
        iqs = [int(iq)] if isinstance(iq, int) else [int(x) for x in iq]
        om = [float(w) for w in omega]
        nw = len(om)
        tot = sum(nw * self.ng[q] ** 2 for q in iqs)
        if out is None:
            out = torch.empty(tot, dtype=torch.complex128, device=f"cuda:{self.device}")
        assert out.dtype == torch.complex128 and out.is_contiguous() and out.numel() >= tot
        dg = torch.empty(sum(nw * self.ng[q] for q in iqs), dtype=torch.float64,
                         device=f"cuda:{self.device}") if diag else None
        iq_arr = (ctypes.c_int * len(iqs))(*iqs)
        om_arr = (ctypes.c_double * nw)(*om)
        self._use_current_stream()
        fn = self.lib.gw_chi0_compute_batch if _batch else self.lib.gw_chi0_compute
        self._check(fn(self.h, len(iqs), iq_arr, nw, om_arr, _ptr(out), _ptr(dg)))
        res, dres, off, doff = [], [], 0, 0
        for q in iqs:
            n = self.ng[q]
            res.append(out[off:off + nw * n * n].view(nw, n, n))
            if diag:
                dres.append(dg[doff:doff + nw * n].view(nw, n))
            off += nw * n * n
            doff += nw * n
        return (res, dres) if diag else res

    def pair_elements(self, iq: int, begin: int, count: int, out: torch.Tensor | None = None):
        n = self.ng[iq]
        if out is None:
            out = torch.empty((count, n), dtype=torch.complex128, device=f"cuda:{self.device}")
        self._use_current_stream()
        self._check(self.lib.gw_chi0_pair_elements(self.h, int(iq), int(begin), int(count), _ptr(out)))
        return out

    def pair_elements_block(self, iq: int, c0: int, cb: int, out: torch.Tensor | None = None):
        """M rows [(c - c0) nv + v] of all valence bands x conduction bands c0 .. c0 + cb - 1 on the
        tensor-core route of stage (a) (gw_chi0_pair_elements_block)."""
        n, nv = self.ng[iq], self.nb[("v", iq)]
        if out is None:
            out = torch.empty((cb * nv, n), dtype=torch.complex128, device=f"cuda:{self.device}")
        self._use_current_stream()
        self._check(self.lib.gw_chi0_pair_elements_block(self.h, int(iq), int(c0), int(cb), _ptr(out)))
        return out

    def contract(self, ev: torch.Tensor, ec: torch.Tensor, M: torch.Tensor, omega: Sequence[float],
                 out: torch.Tensor | None = None):
        ev = ev.to(device=f"cuda:{self.device}", dtype=torch.float64).contiguous()
        ec = ec.to(device=f"cuda:{self.device}", dtype=torch.float64).contiguous()
        M = M.to(device=f"cuda:{self.device}", dtype=torch.complex128).contiguous()
        ng = M.shape[1]
        nw = len(omega)
        if out is None:
            out = torch.empty((nw, ng, ng), dtype=torch.complex128, device=f"cuda:{self.device}")
        om_arr = (ctypes.c_double * nw)(*[float(w) for w in omega])
        self._use_current_stream()
        self._check(self.lib.gw_chi0_contract(self.h, ev.shape[0], ec.shape[0], _ptr(ev), _ptr(ec), ng, _ptr(M),
                                              nw, om_arr, _ptr(out)))
        return out

    def adjoint(self, iq: int, W: torch.Tensor, omega: float = 0.0, want_L: bool = True):
        W = W.to(device=f"cuda:{self.device}", dtype=torch.complex128).contiguous()
        dev = f"cuda:{self.device}"
        nv, nc = self.nb[("v", iq)], self.nb[("c",)]
        dEv = torch.empty(nv, dtype=torch.float64, device=dev)
        dEc = torch.empty(nc, dtype=torch.float64, device=dev)
        dcv = torch.empty((nv, self.ngpsi[("v", iq)]), dtype=torch.complex128, device=dev)
        dcc = torch.empty((nc, self.ngpsi[("c",)]), dtype=torch.complex128, device=dev)
        L = ctypes.c_double(0.0)
        self._use_current_stream()
        self._check(self.lib.gw_chi0_adjoint(self.h, int(iq), float(omega), _ptr(W),
                                             ctypes.byref(L) if want_L else None, _ptr(dEv), _ptr(dEc),
                                             _ptr(dcv), _ptr(dcc)))
        return (L.value if want_L else None), dEv, dEc, dcv, dcc

    def subspace_basis(self, chi0: torch.Tensor, neig: int):
        """C_s [ng, neig] and the neig most negative eigenvalues of a Hermitian chi(0) block."""
        chi0 = chi0.to(device=f"cuda:{self.device}", dtype=torch.complex128).contiguous()
        ng = chi0.shape[0]
        basis = torch.empty((ng, int(neig)), dtype=torch.complex128, device=f"cuda:{self.device}")
        evals = torch.empty(int(neig), dtype=torch.float64, device=f"cuda:{self.device}")
        self._use_current_stream()
        self._check(self.lib.gw_chi0_subspace_basis(self.h, ng, _ptr(chi0), int(neig), _ptr(basis), _ptr(evals)))
        return basis, evals

    def compute_subspace(self, iq: int, basis: torch.Tensor, omega: Sequence[float], out: torch.Tensor | None = None):
        """chi_BB'(i w) = C_s^H chi(i w) C_s from the projected pair elements: [nw, neig, neig]."""
        basis = basis.to(device=f"cuda:{self.device}", dtype=torch.complex128).contiguous()
        neig = basis.shape[1]
        nw = len(omega)
        if out is None:
            out = torch.empty((nw, neig, neig), dtype=torch.complex128, device=f"cuda:{self.device}")
        om_arr = (ctypes.c_double * nw)(*[float(w) for w in omega])
        self._use_current_stream()
        self._check(self.lib.gw_chi0_compute_subspace(self.h, int(iq), neig, _ptr(basis), nw, om_arr, _ptr(out)))
        return out

    def jvp(self, iq: int, omega: Sequence[float], dcv: torch.Tensor, dcc: torch.Tensor, dEv: torch.Tensor,
            dEc: torch.Tensor, out: torch.Tensor | None = None):
        """d chi0 [nw, ng, ng] along tangent coefficients (dcv [nv, ngpsi_v], dcc [nc, ngpsi_c]) and
        tangent energies (dEv [nv], dEc [nc])."""
        dev = f"cuda:{self.device}"
        args = [t.to(device=dev, dtype=dt).contiguous() for t, dt in
                ((dcv, torch.complex128), (dcc, torch.complex128), (dEv, torch.float64), (dEc, torch.float64))]
        n = self.ng[int(iq)]
        nw = len(omega)
        if out is None:
            out = torch.empty((nw, n, n), dtype=torch.complex128, device=dev)
        om_arr = (ctypes.c_double * nw)(*[float(w) for w in omega])
        self._use_current_stream()
        self._check(self.lib.gw_chi0_jvp(self.h, int(iq), nw, om_arr, *[_ptr(a) for a in args], _ptr(out)))
        return out

    def compute_real(self, iq: int, omega: Sequence[float], eta: float, out: torch.Tensor | None = None):
        """chi0 on the real axis with broadening eta: [nw, ng, ng] complex (not Hermitian)."""
        n = self.ng[int(iq)]
        nw = len(omega)
        if out is None:
            out = torch.empty((nw, n, n), dtype=torch.complex128, device=f"cuda:{self.device}")
        om_arr = (ctypes.c_double * nw)(*[float(w) for w in omega])
        self._use_current_stream()
        self._check(self.lib.gw_chi0_compute_real(self.h, int(iq), nw, om_arr, float(eta), _ptr(out)))
        return out

    def epsilon_inverse(self, chi: torch.Tensor, vcoul: torch.Tensor, out: torch.Tensor | None = None):
        """[I - v chi(w)]^-1 for chi blocks [nw, ng, ng] (or [ng, ng]) and v [ng]."""
        chi = chi.to(device=f"cuda:{self.device}", dtype=torch.complex128).contiguous()
        single = chi.dim() == 2
        chi = chi.view(-1, chi.shape[-2], chi.shape[-1])
        nw, ng = chi.shape[0], chi.shape[1]
        v = vcoul.to(device=f"cuda:{self.device}", dtype=torch.float64).contiguous()
        if out is None:
            out = torch.empty_like(chi)
        self._use_current_stream()
        self._check(self.lib.gw_chi0_epsilon_inverse(self.h, ng, nw, _ptr(chi), _ptr(v), _ptr(out)))
        return out[0] if single else out

    def sigma_gpp(self, M: torch.Tensor, En, nocc: int, omega2: torch.Tensor, wtilde: torch.Tensor,
                  vcoul: torch.Tensor, E, out: torch.Tensor | None = None):
        """Full self-energy matrix of the plasmon-pole model on the energy grid E:
        M [nb, nsig, ng] (M[n][l][G]), En [nb] (host), the first nocc bands occupied, Omega^2 and
        mode energies [ng, ng], v [ng].  Returns [ne, nsig, nsig] complex128."""
        dev = f"cuda:{self.device}"
        M = M.to(device=dev, dtype=torch.complex128).contiguous()
        nb, nsig, ng = M.shape
        o2 = omega2.to(device=dev, dtype=torch.complex128).contiguous()
        wt = wtilde.to(device=dev, dtype=torch.complex128).contiguous()
        v = vcoul.to(device=dev, dtype=torch.float64).contiguous()
        en = [float(x) for x in En]
        ee = [float(x) for x in E]
        if len(en) != nb:
            raise ValueError("En must have one energy per band")
        ne = len(ee)
        if out is None:
            out = torch.empty((ne, nsig, nsig), dtype=torch.complex128, device=dev)
        en_arr = (ctypes.c_double * max(nb, 1))(*en)
        e_arr = (ctypes.c_double * max(ne, 1))(*ee)
        self._use_current_stream()
        self._check(self.lib.gw_chi0_sigma_gpp(self.h, nb, int(nocc), nsig, ng, _ptr(M), en_arr, _ptr(o2), _ptr(wt),
                                               _ptr(v), ne, e_arr, _ptr(out)))
        return out

    def keep_pair_elements(self, enable: bool = True):
        """Keep the pair elements of the last computed slot resident for compute_subspace and
        compute_real on that slot (P x N_G complex128 of device memory)."""
        self._check(self.lib.gw_chi0_keep_pair_elements(self.h, 1 if enable else 0))

    def streams(self, iq: int = 0) -> int:
        """Streams compute() uses for slot iq: 2 with the contraction beside the pair kernel, else 1."""
        r = int(self.lib.gw_chi0_streams(self.h, int(iq)))
        if r < 0:
            raise GwError(-r, self.lib.gw_chi0_last_error(self.h).decode())
        return r

    def sync(self):
        self._use_current_stream()
        self._check(self.lib.gw_chi0_sync(self.h))

    def set_timing(self, enable: bool):
        self._check(self.lib.gw_chi0_set_timing(self.h, 1 if enable else 0))

    def timing(self, reset: bool = True):
        n = 32
        names = (ctypes.c_char * 32 * n)()
        ms = (ctypes.c_double * n)()
        cnt = (ctypes.c_int64 * n)()
        k = self.lib.gw_chi0_timing(self.h, n, names, ms, cnt, 1 if reset else 0)
        return {bytes(names[i]).split(b"\0")[0].decode(): (ms[i], cnt[i]) for i in range(min(k, n))}

    def device_bytes(self) -> int:
        return int(self.lib.gw_chi0_device_bytes(self.h))

    def destroy(self):
        if getattr(self, "h", None):
            self.lib.gw_chi0_destroy(self.h)
            self.h = None

    close = destroy

    def __del__(self):
        try:
            self.destroy()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.destroy()


def contract_noalloc(ev: torch.Tensor, ec: torch.Tensor, M: torch.Tensor, omega: Sequence[float],
                     out: torch.Tensor) -> torch.Tensor:
    """FP64 contraction through gw_chi0_contract_noalloc: no device allocation inside the call.

    For callers that cannot allocate device memory (a host framework that owns every
    allocation through its own pool, or a hot path where allocator calls are forbidden).
    All tensors must already be on the current device, contiguous: float64 ev [nv] and
    ec [nc], complex128 M [nv*nc, ng], complex128 out [nw, ng, ng] (1 <= nw <= 64).  The
    call uses the library's fixed scratch array, so calls must not overlap on the GPU.
    Raises ValueError before anything reaches the library when a tensor does not match.
    """
    nw = len(omega)
    cur = torch.device("cuda", torch.cuda.current_device()) if torch.cuda.is_available() else None
    for name, t, dt in (("ev", ev, torch.float64), ("ec", ec, torch.float64), ("M", M, torch.complex128),
                        ("out", out, torch.complex128)):
        if not isinstance(t, torch.Tensor) or cur is None or t.device != cur:
            raise ValueError(f"{name} must be a tensor on the current CUDA device")
        if t.dtype != dt:
            raise ValueError(f"{name} must be {dt}, got {t.dtype}")
        if not t.is_contiguous():
            raise ValueError(f"{name} must be contiguous")
    if ev.dim() != 1 or ec.dim() != 1 or M.dim() != 2:
        raise ValueError("ev, ec must be 1-D and M 2-D")
    if not 1 <= nw <= 64:
        raise ValueError("need 1 <= len(omega) <= 64")
    ng = M.shape[1]
    if M.shape[0] != ev.numel() * ec.numel():
        raise ValueError(f"M has {M.shape[0]} rows, expected nv * nc = {ev.numel() * ec.numel()}")
    if tuple(out.shape) != (nw, ng, ng):
        raise ValueError(f"out must have shape {(nw, ng, ng)}, got {tuple(out.shape)}")
    lib = _lib.load()
    om_arr = (ctypes.c_double * nw)(*[float(w) for w in omega])
    st = lib.gw_chi0_contract_noalloc(ev.shape[0], ec.shape[0], _ptr(ev), _ptr(ec), M.shape[1], _ptr(M), nw,
                                      om_arr, _ptr(out), _stream_handle())
    if st != 0:
        raise GwError(st, "gw_chi0_contract_noalloc failed")
    return out


class Chi0Fn(torch.autograd.Function):
    """chi0(iw) of one q-point as a differentiable function of the band coefficients and energies.

    forward(handle, gvec, cv, ev, cc, ec, gchi, omega) loads the bands into slot 0 of
    ``handle`` and returns chi [ng, ng] (complex128).  backward receives dL/dchi for a
    real L and passes it unchanged to gw_chi0_adjoint, which uses its Hermitian part W (chi is
    Hermitian, so L = Re Tr(W chi) locally) and returns the gradients (torch's
    convention for complex inputs: dL/dRe + i dL/dIm).
    """

    @staticmethod
    def forward(ctx, handle, gvec, cv, ev, cc, ec, gchi, omega):
        handle.set_bands(0, 1, gvec, cc.detach(), ec.detach())
        handle.set_bands(0, 0, gvec, cv.detach(), ev.detach())
        handle.set_gsphere(0, gchi)
        (chi,) = handle.compute(0, [float(omega)])
        ctx.handle, ctx.omega = handle, float(omega)
        return chi[0].clone()

    @staticmethod
    def backward(ctx, gchi_out):
        # the library takes the Hermitian part of the upstream gradient itself
        _, dEv, dEc, dcv, dcc = ctx.handle.adjoint(0, gchi_out.contiguous(), omega=ctx.omega, want_L=False)
        return None, None, dcv, dEv, dcc, dEc, None, None


def create(grid, **kw) -> Chi0:
    return Chi0(grid, **kw)


def from_problem(prob, prec: str = "fp64", nslices: int = 6, pair_chunk: int = 8192, **kw) -> Chi0:
    """Handle with one q slot loaded from a gwgen.Problem (inputs copied to the GPU)."""
    dev = torch.device("cuda", torch.cuda.current_device())
    h = Chi0(prob.grid, nq=1, prec=prec, nslices=nslices, pair_chunk=pair_chunk, **kw)
    g = torch.as_tensor(prob.gpsi, device=dev)
    h.set_bands(0, 1, g, torch.as_tensor(prob.cc, device=dev), torch.as_tensor(prob.ec, device=dev))
    h.set_bands(0, 0, g, torch.as_tensor(prob.cv, device=dev), torch.as_tensor(prob.ev, device=dev))
    h.set_gsphere(0, torch.as_tensor(prob.gchi, device=dev))
    return h
