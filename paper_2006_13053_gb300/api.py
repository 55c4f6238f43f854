"""Python face of the CUDA library: thin wrappers that pass torch device tensors to the C ABI.

    plan = Plan(cand, s, precision=FP32, refine=1, tau_abs=...)   # cand: int32 cuda [n, d]
    supp, coef = plan.reconstruct(samples)                         # samples: complex cuda [sum M]

All arithmetic runs in libsfft.so; no step falls back to PyTorch or the CPU.
"""
from __future__ import annotations

import ctypes as C

import numpy as np
import torch

from . import _native as N


def _ptr(t):
    return None if t is None else C.c_void_p(t.data_ptr())


def _stream(stream=None):
    s = stream if stream is not None else torch.cuda.current_stream()
    return C.c_void_p(s.cuda_stream)


def _req(t, dtype, name):
    if not (isinstance(t, torch.Tensor) and t.is_cuda and t.dtype == dtype and t.is_contiguous()):
        raise TypeError(f"{name} must be a contiguous CUDA tensor of dtype {dtype}")
    return t


class Plan:
    """A reconstruction plan (Algorithm 2/4) over the candidate set `cand` (kept referenced)."""

    def __init__(self, cand: torch.Tensor, s: int, L: int = 0, M=None, z=None, stream=None, d=None, **params):
        """cand: int32 [n, d], or int8 [n, ld] rows (|k_t| <= 127, ld >= d, the first d bytes of a
        row are the frequency, the tensor 4-byte aligned; pass d)."""
        if not (isinstance(cand, torch.Tensor) and cand.dim() == 2):
            raise ValueError("cand must be a 2-D tensor [n, d] (int32) or [n, ld] (int8)")
        if cand.dtype == torch.int8:
            _req(cand, torch.int8, "cand")
            if d is None:
                raise ValueError("int8 candidate rows need d")
            params.setdefault("cand_type", N.CAND_I8)
            params.setdefault("cand_ld", int(cand.shape[1]))
            self.n, self.d = int(cand.shape[0]), int(d)
        else:
            _req(cand, torch.int32, "cand")
            self.n, self.d = cand.shape
            if d is not None and d != self.d:
                raise ValueError("d does not match the int32 rows")
        self.cand = cand
        self.params = N.default_params(**params)
        self.stream = stream
        Mp = zp = None
        if M is not None:
            M = np.ascontiguousarray(np.broadcast_to(np.asarray(M, dtype=np.int64), (L,)))
            Mp = M.ctypes.data_as(C.c_void_p)
        if z is not None:
            z = np.ascontiguousarray(np.asarray(z, dtype=np.int64))
            zp = z.ctypes.data_as(C.c_void_p)
        h = C.c_void_p()
        N.check(N.sfft_plan_create(C.byref(h), self.d, C.c_void_p(cand.data_ptr()), self.n, int(s), int(L), Mp, zp,
                                   C.byref(self.params), _stream(stream)))
        self.handle = h
        Lr = C.c_int()
        ns = C.c_int64()
        N.check(N.sfft_plan_info(h, C.byref(Lr), None, None, C.byref(ns)))
        self.L = Lr.value
        self.n_samples = ns.value
        Ma = np.zeros(self.L, dtype=np.int64)
        za = np.zeros(self.L * self.d, dtype=np.int64)
        N.check(N.sfft_plan_info(h, None, Ma.ctypes.data_as(C.c_void_p), za.ctypes.data_as(C.c_void_p), None))
        self.M = Ma
        self.z = za.reshape(self.L, self.d)
        self.offsets = np.concatenate([[0], np.cumsum(Ma)]).astype(np.int64)
        self.cdtype = torch.complex64 if self.params.precision == N.FP32 else torch.complex128
        self.last_nout = 0

    def close(self):
        if getattr(self, "handle", None):
            N.sfft_plan_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def set_candidates(self, cand):
        """Rebind to another candidate set of the same layout (at most the creation size, |k_t|
        within the creation bound); kept referenced like the first one."""
        if cand.dtype != self.cand.dtype or cand.dim() != 2 or cand.shape[1] != self.cand.shape[1]:
            raise ValueError("the new candidate rows need the plan's dtype and row width")
        _req(cand, cand.dtype, "cand")
        N.check(N.sfft_plan_set_candidates(self.handle, C.c_void_p(cand.data_ptr()), int(cand.shape[0])))
        self.cand = cand
        self.n = int(cand.shape[0])

    def set_generators(self, z):
        """New generating vectors (int [L, d], 0 <= z < M_l) on the same lattice sizes."""
        z = np.ascontiguousarray(np.asarray(z, dtype=np.int64).reshape(self.L, self.d))
        N.check(N.sfft_plan_set_generators(self.handle, z.ctypes.data_as(C.c_void_p)))
        self.z = z.copy()

    # ---------------------------------------------------------------- nodes and samplers
    def sample_points(self):
        """(numerators int32 [sum M, d], x float64 [sum M, d]) of eq. (2.1)."""
        dev = self.cand.device
        num = torch.empty((self.n_samples, self.d), dtype=torch.int32, device=dev)
        x = torch.empty((self.n_samples, self.d), dtype=torch.float64, device=dev)
        N.check(N.sfft_sample_points(self.handle, _ptr(num), _ptr(x), None))
        return num, x

    def sample_sparse_poly(self, kvec, coef, noise=None, out=None):
        _req(kvec, torch.int32, "kvec")
        _req(coef, torch.complex128, "coef")
        if noise is not None:
            _req(noise, self.cdtype, "noise")  # complex in the plan precision
        out = out if out is not None else torch.empty(self.n_samples, dtype=self.cdtype, device=self.cand.device)
        N.check(N.sfft_sample_sparse_poly(self.handle, _ptr(kvec), _ptr(coef), kvec.shape[0], _ptr(noise), _ptr(out)))
        return out

    def sample_sop(self, triples, theta, K=48, width=32.0, out=None):
        tri = np.ascontiguousarray(np.asarray(triples, dtype=np.int32))
        _req(theta, torch.float64, "theta")
        out = out if out is not None else torch.empty(self.n_samples, dtype=self.cdtype, device=self.cand.device)
        N.check(N.sfft_sample_sop(self.handle, tri.ctypes.data_as(C.c_void_p), _ptr(theta), tri.shape[0], K,
                                  float(width), _ptr(out)))
        return out

    def sample_bspline(self, terms, out=None):
        """Section 4.3's test function (eq. 4.3) at the lattice nodes: terms = [(dims, m), ...],
        f(x) = sum over terms of prod_{t in dims} N_m(x_t) (periodic B-splines, unit L2 norm)."""
        dims = np.full((len(terms), 4), -1, dtype=np.int32)
        orders = np.zeros(len(terms), dtype=np.int32)
        for q, (dq, m) in enumerate(terms):
            if len(dq) > 4:
                raise ValueError("a B-spline term acts on at most 4 dimensions")
            dims[q, :len(dq)] = dq
            orders[q] = m
        out = out if out is not None else torch.empty(self.n_samples, dtype=self.cdtype, device=self.cand.device)
        N.check(N.sfft_sample_bspline(self.handle, dims.ctypes.data_as(C.c_void_p), orders.ctypes.data_as(C.c_void_p),
                                      len(terms), _ptr(out)))
        return out

    def sample_sop_backward(self, triples, theta, dsamples, K=48, width=32.0):
        tri = np.ascontiguousarray(np.asarray(triples, dtype=np.int32))
        _req(theta, torch.float64, "theta")
        _req(dsamples, self.cdtype, "dsamples")
        dtheta = torch.empty(tri.shape[0], dtype=torch.float64, device=self.cand.device)
        N.check(N.sfft_sample_sop_backward(self.handle, tri.ctypes.data_as(C.c_void_p), _ptr(theta), tri.shape[0], K,
                                           float(width), _ptr(dsamples), _ptr(dtheta)))
        return dtheta

    # ---------------------------------------------------------------- reconstruction
    def reconstruct(self, samples, cap=None, diag=False, counts=False, hashes=False, collisions=False):
        """Returns (supp int64 [k], coef complex128 [k]) and, with diag=True, a dict of diagnostics."""
        _req(samples, self.cdtype, "samples")
        dev = self.cand.device
        cap = int(cap if cap is not None else max(self.params.s_tilde or 0, 1) + 4 * 4096)
        supp = torch.empty(cap, dtype=torch.int64, device=dev)
        coef = torch.empty(cap, dtype=torch.complex128, device=dev)
        nout = C.c_int64()
        D = None
        info = {}
        if diag or counts or hashes or collisions:
            D = N.Diag()
            dcap = self.n  # >= the plan's detected-set capacity
            info["detected_buf"] = torch.empty(dcap, dtype=torch.int64, device=dev)
            info["pcheck_buf"] = torch.empty(dcap, dtype=torch.complex128, device=dev)
            info["ghat"] = torch.empty(self.n_samples, dtype=torch.complex128, device=dev)
            info["tau"] = torch.empty(self.L, dtype=torch.float64, device=dev)
            D.detected = info["detected_buf"].data_ptr()
            D.pcheck = info["pcheck_buf"].data_ptr()
            D.ghat = info["ghat"].data_ptr()
            D.tau = info["tau"].data_ptr()
            if counts:
                info["counts"] = torch.empty(self.n, dtype=torch.uint8, device=dev)
                D.counts = info["counts"].data_ptr()
            if hashes:
                info["hashes"] = torch.empty((self.n, self.L), dtype=torch.int32, device=dev)
                D.hashes = info["hashes"].data_ptr()
            if collisions:
                info["collisions"] = torch.empty(self.n_samples, dtype=torch.int32, device=dev)
                D.collisions = info["collisions"].data_ptr()
        rc = N.sfft_reconstruct(self.handle, _ptr(samples), _ptr(supp), _ptr(coef), cap, C.byref(nout),
                                C.byref(D) if D is not None else None)
        N.check(rc)
        k = nout.value
        self.last_nout = k
        if D is not None:
            nd = D.n_detected
            info["n_detected"] = nd
            info["n_guard"] = D.n_guard
            info["lsq_iters"] = D.lsq_iters
            info["detected"] = info.pop("detected_buf")[:nd]
            info["pcheck"] = info.pop("pcheck_buf")[:nd]
            return supp[:k], coef[:k], info
        return supp[:k], coef[:k]

    def shard_begin(self, samples):
        """First half of a sharded reconstruction: this plan's slice through the median combine;
        returns C (complex128 cuda [sum M]), the slice's median coefficients in their buckets."""
        _req(samples, self.cdtype, "samples")
        C_ = torch.empty(self.n_samples, dtype=torch.complex128, device=self.cand.device)
        nd = C.c_int64()
        N.check(N.sfft_reconstruct_shard_begin(self.handle, _ptr(samples), _ptr(C_), C.byref(nd)))
        self.shard_detected = nd.value
        return C_

    def shard_end(self, C_sum, cap=None):
        """Second half: refinement with the summed C, Algorithm 4 on the slice.  Returns (supp into
        the slice, coef, rank keys as int64 tensors of the key bits)."""
        _req(C_sum, torch.complex128, "C_sum")
        dev = self.cand.device
        cap = int(cap if cap is not None else max(self.params.s_tilde or 0, 1) + 4 * 4096)
        supp = torch.empty(cap, dtype=torch.int64, device=dev)
        coef = torch.empty(cap, dtype=torch.complex128, device=dev)
        keys = torch.empty(cap, dtype=torch.int64, device=dev)  # uint64 bits (keys of moduli < 2^63)
        nout = C.c_int64()
        N.check(N.sfft_reconstruct_shard_end(self.handle, _ptr(C_sum), _ptr(supp), _ptr(coef), _ptr(keys), cap,
                                             C.byref(nout)))
        k = nout.value
        return supp[:k], coef[:k], keys[:k]

    def backward(self, dcoef):
        """Sample cotangents for coefficient cotangents of the last reconstruct (support fixed)."""
        _req(dcoef, torch.complex128, "dcoef")
        if dcoef.shape[0] != self.last_nout:
            raise ValueError("dcoef must match the last reconstruct's output size")
        ds = torch.empty(self.n_samples, dtype=self.cdtype, device=self.cand.device)
        N.check(N.sfft_reconstruct_backward(self.handle, _ptr(dcoef), _ptr(ds)))
        return ds


class SopReconstruct(torch.autograd.Function):
    """theta -> samples of the sum-of-products function at the plan's lattice nodes ->
    reconstructed coefficients on the selected support.  The backward pass runs the adjoint
    kernels (coefficient cotangents -> buckets -> inverse prime-length FFT -> samples -> theta),
    recomputing the samples' factors instead of storing them."""

    @staticmethod
    def forward(ctx, theta, plan, triples, K, width):
        samples = plan.sample_sop(triples, theta, K=K, width=width)
        supp, coef = plan.reconstruct(samples)
        ctx.plan, ctx.triples, ctx.K, ctx.width = plan, triples, K, width
        ctx.save_for_backward(theta)
        ctx.mark_non_differentiable(supp)
        return supp, coef

    @staticmethod
    def backward(ctx, gsupp, gcoef):
        (theta,) = ctx.saved_tensors
        plan = ctx.plan
        if gcoef is None:
            return None, None, None, None, None
        # torch's complex gradient convention for a real loss is dL/dRe + i dL/dIm
        ds = plan.backward(gcoef.contiguous().to(torch.complex128))
        dtheta = plan.sample_sop_backward(ctx.triples, theta, ds, K=ctx.K, width=ctx.width)
        return dtheta, None, None, None, None


class Batch:
    """Several plans (same precision) reconstructed with one launch per stage; with
    use_graph=True the stage sequence is captured once into a CUDA graph and replayed.
    Output buffers are allocated once so that their addresses stay fixed."""

    def __init__(self, plans, use_graph=False, stream=None, caps=None):
        self.plans = list(plans)
        self.stream = stream
        n = len(self.plans)
        arr = (C.c_void_p * n)(*[p.handle.value for p in self.plans])
        h = C.c_void_p()
        N.check(N.sfft_batch_create(C.byref(h), arr, n, 1 if use_graph else 0, _stream(stream)))
        self.handle = h
        dev = self.plans[0].cand.device
        self.caps = [int(c) for c in (caps or [max(p.params.s_tilde or 0, 1) + 4 * 4096 for p in self.plans])]
        # one buffer for all supports and one for all coefficients (a result read-back is one copy
        # each); self.supp / self.coef hold the per-plan views
        self.supp_all = torch.empty(sum(self.caps), dtype=torch.int64, device=dev)
        self.coef_all = torch.empty(sum(self.caps), dtype=torch.complex128, device=dev)
        offs = np.concatenate([[0], np.cumsum(self.caps)]).astype(np.int64)
        self.supp = [self.supp_all[offs[i]:offs[i + 1]] for i in range(n)]
        self.coef = [self.coef_all[offs[i]:offs[i + 1]] for i in range(n)]
        self.nout = torch.zeros(n, dtype=torch.int64, device=dev)
        self._ps = (C.c_void_p * n)(*[t.data_ptr() for t in self.supp])
        self._pc = (C.c_void_p * n)(*[t.data_ptr() for t in self.coef])
        self._cap = (C.c_int64 * n)(*self.caps)

    def reconstruct_async(self, samples):
        """Enqueue every reconstruction; results stay in self.supp / self.coef / self.nout."""
        n = len(self.plans)
        for p, s in zip(self.plans, samples):
            _req(s, p.cdtype, "samples")
        sp = (C.c_void_p * n)(*[s.data_ptr() for s in samples])
        N.check(N.sfft_batch_reconstruct(self.handle, sp, self._ps, self._pc, self._cap,
                                         C.c_void_p(self.nout.data_ptr())))

    def sample_sparse_poly(self, kvecs, coefs, noises=None, outs=None):
        """Samples of every plan's sparse polynomial (+ noise) in shared launches (asynchronous)."""
        n = len(self.plans)
        outs = outs if outs is not None else [torch.empty(p.n_samples, dtype=p.cdtype, device=p.cand.device)
                                              for p in self.plans]
        for p, k, c, o in zip(self.plans, kvecs, coefs, outs):
            _req(k, torch.int32, "kvec")
            _req(c, torch.complex128, "coef")
            _req(o, p.cdtype, "samples_out")
        kp = (C.c_void_p * n)(*[k.data_ptr() for k in kvecs])
        cp = (C.c_void_p * n)(*[c.data_ptr() for c in coefs])
        nt = (C.c_int64 * n)(*[k.shape[0] for k in kvecs])
        npp = None
        if noises is not None:
            for p, x in zip(self.plans, noises):
                if x is not None:
                    _req(x, p.cdtype, "noise")  # complex in the plan precision
            npp = (C.c_void_p * n)(*[(x.data_ptr() if x is not None else 0) for x in noises])
        op = (C.c_void_p * n)(*[o.data_ptr() for o in outs])
        N.check(N.sfft_batch_sample_sparse_poly(self.handle, kp, cp, nt, npp, op))
        return outs

    def autotune(self, samples, reps=2):
        """Pick the fastest hash grid and transform CTA size on these inputs; returns them."""
        n = len(self.plans)
        sp = (C.c_void_p * n)(*[s.data_ptr() for s in samples])
        hw = C.c_double()
        ft = C.c_int()
        N.check(N.sfft_batch_autotune(self.handle, sp, self._ps, self._pc, self._cap, int(reps), C.byref(hw),
                                      C.byref(ft)))
        return hw.value, ft.value

    def set_shapes(self, hash_waves, fft_threads):
        """Apply launch shapes that autotune() returned (e.g. for a second batch of the same plans'
        shapes); see sfft_batch_set_shapes in the C header."""
        N.check(N.sfft_batch_set_shapes(self.handle, float(hash_waves), int(fft_threads)))

    def select_hash(self, tensor=True):
        """Use the tensor-core hash kernel for the launches that qualify (see the C header)."""
        N.check(N.sfft_batch_select_hash(self.handle, 1 if tensor else 0))

    def launch_count(self):
        """(kernel launches of one reconstruct call, of one sampler call) in the steady state."""
        r, sm = C.c_int(), C.c_int()
        N.check(N.sfft_batch_launch_count(self.handle, C.byref(r), C.byref(sm)))
        return r.value, sm.value

    def flags(self):
        fl = (C.c_int64 * len(self.plans))()
        rc = N.sfft_batch_flags(self.handle, fl)
        return rc, list(fl)

    def results(self, check=True):
        (self.stream or torch.cuda.current_stream()).synchronize()
        if check:
            rc, _ = self.flags()
            N.check(rc)
        k = self.nout.cpu().tolist()
        return [(s[:m], c[:m]) for s, c, m in zip(self.supp, self.coef, k)]

    def reconstruct(self, samples):
        self.reconstruct_async(samples)
        return self.results()

    def timing(self, mode=-1):
        """(mode: 1 enable+reset, 0 disable+reset, -1 read) -> {stage: (ms_total, calls)}."""
        ms = (C.c_double * 12)()
        nl = (C.c_int64 * 12)()
        r = N.sfft_batch_timing(self.handle, int(mode), ms, nl)
        if r < 0:
            raise N.SfftError(N.ECUDA, N.sfft_last_error().decode())
        return {name: (ms[i], nl[i]) for i, name in enumerate(N.STAGES)}

    def close(self):
        if getattr(self, "handle", None):
            N.sfft_batch_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def dim_incremental(d, lo, hi, s, fn, s_local=0, r=1, stream=None, cap=None, **params):
    """Algorithm 3 on the box prod_t [lo_t, hi_t] with a built-in black box:
       fn = ("sparse_poly", kvec int32 cuda [n, d], coef complex128 cuda [n]) or
       fn = ("sop", triples int [m, 3], theta float64 cuda [m], K, width) or
       fn = ("bspline", terms): Section 4.3's B-spline sum, terms = [(dims, order), ...].
    Returns (supp int32 numpy [k, d] in lexicographic order, coef complex128 numpy [k], samples)."""
    p = N.default_dimincr_params(s=int(s), s_local=int(s_local), r=int(r), **params)
    lo = np.ascontiguousarray(np.broadcast_to(np.asarray(lo, dtype=np.int32), (d,)))
    hi = np.ascontiguousarray(np.broadcast_to(np.asarray(hi, dtype=np.int32), (d,)))
    keep = []
    if fn[0] == "sparse_poly":
        _, kvec, coef = fn
        _req(kvec, torch.int32, "kvec")
        _req(coef, torch.complex128, "coef")
        ctx = N.SparsePolyCtx(kvec.data_ptr(), coef.data_ptr(), kvec.shape[0], d)
        faddr = N.fn_address("sfft_fn_sparse_poly")
    elif fn[0] == "sop":
        _, triples, theta, K, width = fn
        tri = np.ascontiguousarray(np.asarray(triples, dtype=np.int32))
        _req(theta, torch.float64, "theta")
        m = tri.shape[0]
        work = torch.empty(16 * m * (K + 1) + 12 * m + 64, dtype=torch.uint8, device=theta.device)
        keep += [tri, work]
        ctx = N.SopCtx(tri.ctypes.data_as(C.c_void_p).value, theta.data_ptr(), m, int(K), float(width), d,
                       work.data_ptr())
        faddr = N.fn_address("sfft_fn_sop")
    elif fn[0] == "bspline":
        terms = fn[1]
        dims = np.full((len(terms), 4), -1, dtype=np.int32)
        orders = np.zeros(len(terms), dtype=np.int32)
        for q, (dq, m) in enumerate(terms):
            dims[q, :len(dq)] = dq
            orders[q] = m
        keep += [dims, orders]
        ctx = N.BsplineCtx(dims.ctypes.data_as(C.c_void_p).value, orders.ctypes.data_as(C.c_void_p).value,
                           len(terms), d)
        faddr = N.fn_address("sfft_fn_bspline")
    else:
        raise ValueError(fn[0])
    cap = int(cap if cap is not None else s)
    supp = np.zeros((cap, d), dtype=np.int32)
    coefo = np.zeros(cap, dtype=np.complex128)
    nout = C.c_int64()
    nsamp = C.c_int64()
    N.check(N.sfft_dim_incremental(d, lo.ctypes.data_as(C.c_void_p), hi.ctypes.data_as(C.c_void_p), C.byref(p),
                                   C.c_void_p(faddr), C.byref(ctx), supp.ctypes.data_as(C.c_void_p),
                                   coefo.ctypes.data_as(C.c_void_p), cap, C.byref(nout), C.byref(nsamp),
                                   _stream(stream)))
    k = nout.value
    return supp[:k], coefo[:k], nsamp.value
