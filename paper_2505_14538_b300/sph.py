"""Thin PyTorch binding of the C ABI (``include/swift_gpu.h``).

Every method marshals torch CUDA tensors into the pointers the C call takes
and passes the current CUDA stream; every step of the computation runs in
the library's kernels. PyTorch only allocates device memory and owns
streams. Names follow the C entry points (``swift_gpu_<name>`` -> ``<name>``).
"""
from __future__ import annotations

import ctypes
from typing import Optional

import torch

from . import _lib

_F32 = torch.float32


class SwiftGPUError(RuntimeError):
    def __init__(self, code: int, where: str, detail: int = 0):
        self.code = code
        self.detail = detail
        super().__init__(f"{where}: {_lib.ERR_NAMES.get(code, code)} (detail {detail})")


def _check(rc: int, where: str):
    if rc != _lib.OK:
        raise SwiftGPUError(rc, where)


def _ptr(t: Optional[torch.Tensor], dtype=None, cols=None, n=None, name="tensor"):
    if t is None:
        return None
    if not t.is_cuda:
        raise ValueError(f"{name} must be a CUDA tensor")
    if not t.is_contiguous():
        raise ValueError(f"{name} must be contiguous")
    if dtype is not None and t.dtype != dtype:
        raise ValueError(f"{name} must be {dtype}, got {t.dtype}")
    if n is not None and t.shape[0] != n:
        raise ValueError(f"{name} must have {n} rows, got {t.shape[0]}")
    if cols is not None and (t.dim() != 2 or t.shape[1] != cols):
        raise ValueError(f"{name} must have shape (n, {cols})")
    return ctypes.c_void_p(t.data_ptr())


def _stream(stream=None):
    s = stream if stream is not None else torch.cuda.current_stream()
    return ctypes.c_void_p(s.cuda_stream)


def make_params(**kw) -> _lib.Params:
    """Library defaults with keyword overrides (box, gamma_eos, eta, kernel_gamma, alpha_v,
    beta_v, alpha_c, h_tol, max_iter, h_max, cell_margin, flags, leaf_max, leaf_margin, kernel).

    ``kernel`` (0 cubic spline, 1 Wendland C2, 2 Wendland C4) also sets
    kernel_gamma to the shape's own H/h unless kernel_gamma is given.
    """
    p = _lib.default_params()
    if "kernel" in kw and "kernel_gamma" not in kw:  # (an unknown kernel is left to the library to refuse)
        kw = dict(kw, kernel_gamma=_lib.KERNEL_GAMMAS.get(int(kw["kernel"]), p.kernel_gamma))
    for k, v in kw.items():
        if k == "box":
            p.box = (ctypes.c_float * 3)(*[float(b) for b in v])
        elif not hasattr(p, k):
            raise KeyError(k)
        else:
            setattr(p, k, v)
    return p


class Context:
    """One library context (``swift_gpu_create``) sized for up to ``n_max`` particles."""

    def __init__(self, n_max: int, **params):
        self.lib = _lib.load()
        self.params = make_params(**params)
        self.n_max = int(n_max)
        self.handle = ctypes.c_void_p()
        _check(self.lib.swift_gpu_create(ctypes.byref(self.handle), ctypes.byref(self.params),
                                         ctypes.c_int64(self.n_max)), "swift_gpu_create")
        self.n = 0
        # count of calls that replace the context's loop state (sorted arrays, sums, ghost records);
        # the autograd functions below compare it to find out whether their forward state is still there
        self.calls = 0

    def close(self):
        if self.handle:
            self.lib.swift_gpu_destroy(self.handle)
            self.handle = ctypes.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def set_params(self, **params):
        self.params = make_params(**{**self._params_dict(), **params})
        _check(self.lib.swift_gpu_set_params(self.handle, ctypes.byref(self.params)), "swift_gpu_set_params")

    def _params_dict(self):
        p = self.params
        return dict(box=tuple(p.box), gamma_eos=p.gamma_eos, eta=p.eta, kernel_gamma=p.kernel_gamma,
                    alpha_v=p.alpha_v, beta_v=p.beta_v, alpha_c=p.alpha_c, h_tol=p.h_tol, max_iter=p.max_iter,
                    h_max=p.h_max, cell_margin=p.cell_margin, flags=p.flags, leaf_max=p.leaf_max,
                    leaf_margin=p.leaf_margin, kernel=p.kernel)

    # ------------------------------------------------------------ calls
    def build_cells(self, pos_h: torch.Tensor, min_cell_width: float = 0.0, stream=None):
        self.calls += 1
        n = pos_h.shape[0]
        _check(self.lib.swift_gpu_build_cells(self.handle, _ptr(pos_h, _F32, 4, name="pos_h"), ctypes.c_int64(n),
                                              ctypes.c_float(min_cell_width), _stream(stream)),
               "swift_gpu_build_cells")
        self.n = n

    def density(self, pos_h, vel_m, active=None, h_out=None, rho4=None, curl_div=None, ngb_count=None,
                want_ngb=True, stream=None):
        self.calls += 1
        n = self.n
        dev = pos_h.device
        if active is not None and (rho4 is None or curl_div is None):
            raise ValueError("with an active subset, rho4 and curl_div carry the inactive particles' values")
        h_out = h_out if h_out is not None else torch.empty(n, dtype=_F32, device=dev)
        rho4 = rho4 if rho4 is not None else torch.empty(n, 4, dtype=_F32, device=dev)
        curl_div = curl_div if curl_div is not None else torch.empty(n, 4, dtype=_F32, device=dev)
        if ngb_count is None and want_ngb:
            ngb_count = torch.zeros(n, dtype=torch.int32, device=dev)
        _check(self.lib.swift_gpu_density(
            self.handle, _ptr(pos_h, _F32, 4, n, "pos_h"), _ptr(vel_m, _F32, 4, n, "vel_m"),
            _ptr(active, torch.uint8, None, n, "active"), _ptr(h_out, _F32, None, n, "h_out"),
            _ptr(rho4, _F32, 4, n, "rho4"), _ptr(curl_div, _F32, 4, n, "curl_div"),
            _ptr(ngb_count, torch.int32, None, n, "ngb_count"), _stream(stream)), "swift_gpu_density")
        return dict(h=h_out, rho4=rho4, curl_div=curl_div, ngb=ngb_count)

    def gradient(self, u, vsig_lapu=None, stream=None):
        self.calls += 1
        n = self.n
        vsig_lapu = vsig_lapu if vsig_lapu is not None else torch.empty(n, 2, dtype=_F32, device=u.device)
        _check(self.lib.swift_gpu_gradient(self.handle, _ptr(u, _F32, None, n, "u"),
                                           _ptr(vsig_lapu, _F32, 2, n, "vsig_lapu"), _stream(stream)),
               "swift_gpu_gradient")
        return vsig_lapu

    def force(self, u, alpha_v=None, alpha_c=None, accel_dudt=None, dh_dt=None, reductions=None,
              want_dh=True, want_reductions=True, stream=None):
        self.calls += 1
        n = self.n
        dev = u.device
        accel_dudt = accel_dudt if accel_dudt is not None else torch.empty(n, 4, dtype=_F32, device=dev)
        if dh_dt is None and want_dh:
            dh_dt = torch.empty(n, dtype=_F32, device=dev)
        if reductions is None and want_reductions:
            reductions = torch.zeros(8, dtype=torch.float64, device=dev)
        _check(self.lib.swift_gpu_force(
            self.handle, _ptr(u, _F32, None, n, "u"), _ptr(alpha_v, _F32, None, n, "alpha_v"),
            _ptr(alpha_c, _F32, None, n, "alpha_c"), _ptr(accel_dudt, _F32, 4, n, "accel_dudt"),
            _ptr(dh_dt, _F32, None, n, "dh_dt"), _ptr(reductions, torch.float64, None, None, "reductions"),
            _stream(stream)), "swift_gpu_force")
        return dict(accel_dudt=accel_dudt, dh_dt=dh_dt, reductions=reductions)

    def gradient_force(self, u, alpha_v=None, alpha_c=None, vsig_lapu=None, accel_dudt=None, dh_dt=None,
                       reductions=None, want_dh=True, want_reductions=True, stream=None):
        """swift_gpu_gradient_force: the outputs of gradient() and force() from one pass over the pairs."""
        self.calls += 1
        n = self.n
        dev = u.device
        vsig_lapu = vsig_lapu if vsig_lapu is not None else torch.empty(n, 2, dtype=_F32, device=dev)
        accel_dudt = accel_dudt if accel_dudt is not None else torch.empty(n, 4, dtype=_F32, device=dev)
        if dh_dt is None and want_dh:
            dh_dt = torch.empty(n, dtype=_F32, device=dev)
        if reductions is None and want_reductions:
            reductions = torch.zeros(8, dtype=torch.float64, device=dev)
        _check(self.lib.swift_gpu_gradient_force(
            self.handle, _ptr(u, _F32, None, n, "u"), _ptr(alpha_v, _F32, None, n, "alpha_v"),
            _ptr(alpha_c, _F32, None, n, "alpha_c"), _ptr(vsig_lapu, _F32, 2, n, "vsig_lapu"),
            _ptr(accel_dudt, _F32, 4, n, "accel_dudt"), _ptr(dh_dt, _F32, None, n, "dh_dt"),
            _ptr(reductions, torch.float64, None, None, "reductions"), _stream(stream)), "swift_gpu_gradient_force")
        return dict(vsig_lapu=vsig_lapu, accel_dudt=accel_dudt, dh_dt=dh_dt, reductions=reductions)

    def force_backward(self, grad_accel_dudt, h_mode: int = 0, stream=None):
        n = self.n
        dev = grad_accel_dudt.device
        gx = torch.empty(n, 4, dtype=_F32, device=dev)
        gv = torch.empty(n, 4, dtype=_F32, device=dev)
        gu = torch.empty(n, dtype=_F32, device=dev)
        _check(self.lib.swift_gpu_force_backward(
            self.handle, _ptr(grad_accel_dudt, _F32, 4, n, "grad_accel_dudt"), _ptr(gx), _ptr(gv), _ptr(gu),
            ctypes.c_int(h_mode), _stream(stream)), "swift_gpu_force_backward")
        return gx, gv, gu

    def set_inactive(self, mask, h, rho4, curl_div, stream=None):
        """swift_gpu_set_inactive: the density results of the particles in ``mask`` computed elsewhere."""
        n = self.n
        self.calls += 1
        _check(self.lib.swift_gpu_set_inactive(
            self.handle, _ptr(mask, torch.uint8, None, n, "mask"), _ptr(h, _F32, None, n, "h"),
            _ptr(rho4, _F32, 4, n, "rho4"), _ptr(curl_div, _F32, 4, n, "curl_div"), _stream(stream)),
            "swift_gpu_set_inactive")

    def sync_status(self):
        code = ctypes.c_int()
        detail = ctypes.c_int64()
        _check(self.lib.swift_gpu_sync_status(self.handle, ctypes.byref(code), ctypes.byref(detail)),
               "swift_gpu_sync_status")
        return code.value, detail.value

    def info(self) -> dict:
        i = _lib.Info()
        _check(self.lib.swift_gpu_get_info(self.handle, ctypes.byref(i)), "swift_gpu_get_info")
        return dict(n=i.n, nc=tuple(i.nc), cell_width=tuple(i.cell_width), h_cap=i.h_cap, n_cells=i.n_cells,
                    n_items=i.n_items, density_passes=i.density_passes, interactions=tuple(i.interactions),
                    candidates=tuple(i.candidates), launches=i.launches, h_iteration_pairs=i.h_iteration_pairs,
                    n_leaves=i.n_leaves, leaf_pairs=i.leaf_pairs, tree_depth=i.tree_depth)

    def leaves(self, stream=None):
        """Adaptive builds: (range (L, 2) int32 sorted [first, end), h_cap (L,), nbr_count (L,)) on the device."""
        nl = self.info()["n_leaves"]
        dev = torch.device("cuda", torch.cuda.current_device())
        rng = torch.empty((nl, 2), dtype=torch.int32, device=dev)
        hcap = torch.empty(nl, dtype=_F32, device=dev)
        cnt = torch.empty(nl, dtype=torch.int32, device=dev)
        if nl:
            _check(self.lib.swift_gpu_get_leaves(self.handle, _ptr(rng), _ptr(hcap), _ptr(cnt), ctypes.c_int64(nl),
                                                 _stream(stream)), "swift_gpu_get_leaves")
        return rng, hcap, cnt

    def cells(self, stream=None):
        n = self.n
        dev = torch.device("cuda", torch.cuda.current_device())
        cid = torch.empty(n, dtype=torch.int32, device=dev)
        perm = torch.empty(n, dtype=torch.int32, device=dev)
        _check(self.lib.swift_gpu_get_cells(self.handle, _ptr(cid), _ptr(perm), _stream(stream)),
               "swift_gpu_get_cells")
        return cid, perm

    def tuning(self) -> dict:
        t = _lib.Tuning()
        _check(self.lib.swift_gpu_get_tuning(self.handle, ctypes.byref(t)), "swift_gpu_get_tuning")
        return dict(threads_per_block=t.threads_per_block, max_lanes_per_particle=t.max_lanes_per_particle,
                    blocks_per_sm=t.blocks_per_sm, wait_limit_us=t.wait_limit_us, group_collect=t.group_collect)

    def set_tuning(self, threads_per_block=None, max_lanes_per_particle=None, blocks_per_sm=None, wait_limit_us=None,
                   group_collect=None):
        """Set the work-distribution knobs; a knob not given keeps its current value.

        max_lanes_per_particle = 1 selects the lane-per-particle path on the uniform grid; 2-32 the cell
        items, whose particles share up to that many lanes of a warp. group_collect picks the
        lane-per-particle path's candidate search: _lib.COLLECT_ROWS (the warp's lanes share the rows of
        cells around them) or _lib.COLLECT_WINDOWS (windows along the 13 pair axes, one lane each)."""
        cur = self.tuning()
        given = dict(threads_per_block=threads_per_block, max_lanes_per_particle=max_lanes_per_particle,
                     blocks_per_sm=blocks_per_sm, wait_limit_us=wait_limit_us, group_collect=group_collect)
        cur.update({k: v for k, v in given.items() if v is not None})
        t = _lib.Tuning(cur["threads_per_block"], cur["max_lanes_per_particle"], cur["blocks_per_sm"],
                        cur["wait_limit_us"], cur["group_collect"])
        _check(self.lib.swift_gpu_set_tuning(self.handle, ctypes.byref(t)), "swift_gpu_set_tuning")

    def autotune(self, loop: int, stream=None):
        self.calls += 1
        _check(self.lib.swift_gpu_autotune(self.handle, ctypes.c_int(loop), _stream(stream)), "swift_gpu_autotune")
        return self.tuning()

    def tune_leaf_max(self, pos_h, vel_m, u, active=None, rho4=None, curl_div=None,
                      candidates=(16, 24, 32, 48, 64), steps=3, stream=None) -> dict:
        """Adaptive contexts: time one step (build_cells, density, fused gradient + force) with each
        leaf_max of ``candidates`` (the median of ``steps`` after one untimed) and keep the fastest.

        pos_h should hold settled h (an earlier step's output), so that no leaf cap is reached; a
        candidate whose step ends with a status other than OK or ERR_H_NOT_CONVERGED is skipped.
        The outputs left in the context are those of the last candidate run: run the step again
        after tuning. Returns {"leaf_max": the choice, "step_ms": {candidate: median ms}}.
        """
        if not self.params.flags & _lib.FLAG_ADAPTIVE:
            raise ValueError("tune_leaf_max needs a context with adaptive leaves")
        s = stream if stream is not None else torch.cuda.current_stream()
        old = int(self.params.leaf_max)
        times = {}
        for lm in candidates:
            self.set_params(leaf_max=int(lm))
            ms = []
            for k in range(steps + 1):
                e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                e0.record(s)
                self.build_cells(pos_h, stream=s)
                self.density(pos_h, vel_m, active, rho4=rho4, curl_div=curl_div, stream=s)
                self.gradient_force(u, stream=s)
                e1.record(s)
                e1.synchronize()
                if k:
                    ms.append(e0.elapsed_time(e1))
            code, _ = self.sync_status()
            if code in (_lib.OK, _lib.ERR_H_NOT_CONVERGED):
                times[int(lm)] = sorted(ms)[len(ms) // 2]
        best = min(times, key=times.get) if times else old
        self.set_params(leaf_max=best)
        return {"leaf_max": best, "step_ms": times}

    # ------------------------------------------------------- whole step
    def density_checked(self, pos_h, vel_m, active=None, rho4=None, curl_div=None, min_cell_width: float = 0.0,
                        check: bool = True, stream=None, **outs):
        """build_cells -> density; with check=True the status word is read (a host synchronisation).

        While the h iteration asks for a support wider than its cap, the
        density call is repeated: on the uniform grid with cells twice as wide
        (up to a third of the box) from the same starting h; with adaptive
        leaves from the capped h, the leaves rebuilt around it (their caps grow
        by 1 + leaf_margin; from the second rebuild on the margin doubles each
        time, up to 4, and the caller's margin is set back afterwards), and
        with wider cells only when h reached the cell cap. ``outs`` are optional output tensors of density() (h_out,
        ngb_count). Raises SwiftGPUError on any status other than OK and
        ERR_H_NOT_CONVERGED.
        """
        self.build_cells(pos_h, min_cell_width, stream)
        d = self.density(pos_h, vel_m, active, rho4=rho4, curl_div=curl_div, stream=stream, **outs)
        if not check:
            return d
        code, detail = self.sync_status()
        box_third = min(float(b) for b in self.params.box) / 3.0
        adaptive = bool(self.params.flags & _lib.FLAG_ADAPTIVE)
        pos_cur = pos_h
        margin = float(self.params.leaf_margin)
        grown = 0
        try:
            for _ in range(32):
                if code != _lib.ERR_H_EXCEEDS_CELL:
                    break
                info = self.info()
                width = max(info["cell_width"])
                if not adaptive or float(d["h"].max()) >= 0.999 * info["h_cap"]:
                    if width >= 0.999 * box_third:
                        break
                    min_w = max(min_cell_width, min(2.0 * width, box_third))
                else:
                    min_w = min_cell_width  # only leaf caps were reached
                    if grown:
                        # a capped h grows by 1 + leaf_margin a rebuild: from the second
                        # rebuild on the margin doubles, so that a far-off h is reached soon
                        self.set_params(leaf_margin=max(margin, min(margin * 2.0 ** grown, 4.0)))
                    grown += 1
                if adaptive:
                    pos_cur = pos_cur.clone()
                    pos_cur[:, 3] = d["h"]
                self.build_cells(pos_cur, min_w, stream)
                d = self.density(pos_cur, vel_m, active, rho4=rho4, curl_div=curl_div, stream=stream, **outs)
                code, detail = self.sync_status()
        finally:
            if float(self.params.leaf_margin) != margin:
                self.set_params(leaf_margin=margin)
        if code not in (_lib.OK, _lib.ERR_H_NOT_CONVERGED):
            raise SwiftGPUError(code, "density", detail)
        d["status"] = (code, detail)
        return d

    def step(self, pos_h, vel_m, u, active=None, rho4=None, curl_div=None, alpha_v=None, alpha_c=None,
             min_cell_width: float = 0.0, check: bool = True, fused: bool = True, stream=None):
        """build_cells -> density (h iteration) -> gradient -> force on one stream.

        fused=True runs gradient and force as one call (swift_gpu_gradient_force,
        the same outputs); fused=False as the two calls. check as in
        density_checked().
        """
        d = self.density_checked(pos_h, vel_m, active, rho4, curl_div, min_cell_width, check, stream)
        out = dict(d)
        if fused:
            out.update(self.gradient_force(u, alpha_v, alpha_c, stream=stream))
        else:
            out["vsig_lapu"] = self.gradient(u, stream=stream)
            out.update(self.force(u, alpha_v, alpha_c, stream=stream))
        return out

    # ------------------------------------------------ time integration (swift_gpu_time.h)
    def kick_drift(self, tp, clock, pos_h, vel_m, u, accel_dudt, dh_dt, vel_pred, u_pred, stream=None):
        n = pos_h.shape[0]
        _check(self.lib.swift_gpu_kick_drift(
            self.handle, ctypes.byref(tp), _ptr(clock, torch.float64, None, 4, "clock"), ctypes.c_int64(n),
            _ptr(pos_h, _F32, 4, n, "pos_h"), _ptr(vel_m, _F32, 4, n, "vel_m"), _ptr(u, _F32, None, n, "u"),
            _ptr(accel_dudt, _F32, 4, n, "accel_dudt"), _ptr(dh_dt, _F32, None, n, "dh_dt"),
            _ptr(vel_pred, _F32, 4, n, "vel_pred"), _ptr(u_pred, _F32, None, n, "u_pred"), _stream(stream)),
            "swift_gpu_kick_drift")

    def viscosity_switch(self, tp, clock, h, u, curl_div, vsig_lapu, div_prev, alpha_v, stream=None):
        n = h.shape[0]
        _check(self.lib.swift_gpu_viscosity_switch(
            self.handle, ctypes.byref(tp), _ptr(clock, torch.float64, None, 4, "clock"), ctypes.c_int64(n),
            _ptr(h, _F32, None, n, "h"), _ptr(u, _F32, None, n, "u"), _ptr(curl_div, _F32, 4, n, "curl_div"),
            _ptr(vsig_lapu, _F32, 2, n, "vsig_lapu"), _ptr(div_prev, _F32, None, n, "div_prev"),
            _ptr(alpha_v, _F32, None, n, "alpha_v"), _stream(stream)), "swift_gpu_viscosity_switch")

    def kick_finish(self, tp, clock, h, pos_h, vel_m, u, accel_dudt, vsig_lapu, alpha_v=None, alpha_c=None,
                    stream=None):
        n = pos_h.shape[0]
        _check(self.lib.swift_gpu_kick_finish(
            self.handle, ctypes.byref(tp), _ptr(clock, torch.float64, None, 4, "clock"), ctypes.c_int64(n),
            _ptr(h, _F32, None, n, "h"), _ptr(pos_h, _F32, 4, n, "pos_h"), _ptr(vel_m, _F32, 4, n, "vel_m"),
            _ptr(u, _F32, None, n, "u"), _ptr(accel_dudt, _F32, 4, n, "accel_dudt"),
            _ptr(vsig_lapu, _F32, 2, n, "vsig_lapu"), _ptr(alpha_v, _F32, None, n, "alpha_v"),
            _ptr(alpha_c, _F32, None, n, "alpha_c"), _stream(stream)), "swift_gpu_kick_finish")


def make_time_params(**kw) -> _lib.TimeParams:
    """Integration defaults (swift_gpu_default_time_params) with keyword overrides."""
    tp = _lib.default_time_params()
    for k, v in kw.items():
        if not hasattr(tp, k):
            raise KeyError(k)
        setattr(tp, k, v)
    return tp


def new_clock(t_end: float = 0.0, device="cuda") -> torch.Tensor:
    """A device swift_gpu_clock (32 bytes as four float64 words): t = 0, dt = dt_next = 0, step 0."""
    c = _lib.Clock(0.0, float(t_end), 0.0, 0.0, 0)
    raw = torch.frombuffer(bytearray(bytes(c)), dtype=torch.float64).clone()
    return raw.to(device)


def read_clock(clock: torch.Tensor) -> dict:
    """Host copy of a device clock (synchronises its stream)."""
    raw = clock.detach().cpu().numpy().tobytes()
    c = _lib.Clock.from_buffer_copy(raw)
    return dict(t=c.t, t_end=c.t_end, dt=c.dt, dt_next=c.dt_next, step=c.step)


class SphForces(torch.autograd.Function):
    """(a, du/dt) = F(x, v, u) at fixed h through the library, differentiable in x, v, u.

    ``forward(x, v, u, m, h, lib_ctx)``: x, v (n, 3), u, m, h (n,) CUDA float32;
    ``lib_ctx`` a :class:`Context` created with ``flags=FLAG_NO_H_ITER`` so the
    given h is used as is. Runs build_cells, density, force. The backward pass
    calls swift_gpu_force_backward (h_mode 0), which reads the context's state
    of this forward call (sorted arrays, sums, ghost records); if the context
    ran other calls in between (its call counter moved), backward first runs
    this forward's calls again from the saved inputs, so the gradient is
    always this forward's.
    """

    @staticmethod
    def forward(ctx, x, v, u, m, h, lib_ctx):
        from . import _lib
        if not (lib_ctx.params.flags & _lib.FLAG_NO_H_ITER):
            raise ValueError("SphForces needs a context created with flags=FLAG_NO_H_ITER (h held fixed)")
        pos_h = torch.cat([x, h[:, None]], 1).float().contiguous()
        vel_m = torch.cat([v, m[:, None]], 1).float().contiguous()
        uu = u.float().contiguous()
        out = SphForces._run(lib_ctx, pos_h, vel_m, uu)
        ctx.lib_ctx = lib_ctx
        ctx.calls = lib_ctx.calls
        ctx.inputs = (pos_h, vel_m, uu)
        ad = out["accel_dudt"]
        return ad[:, :3].clone(), ad[:, 3].clone()

    @staticmethod
    def _run(lib_ctx, pos_h, vel_m, uu):
        lib_ctx.build_cells(pos_h)
        lib_ctx.density(pos_h, vel_m)
        return lib_ctx.force(uu, want_dh=False, want_reductions=False)

    @staticmethod
    def backward(ctx, grad_a, grad_du):
        if ctx.lib_ctx.calls != ctx.calls:  # the context moved on: restore this forward's state
            SphForces._run(ctx.lib_ctx, *ctx.inputs)
        n = ctx.lib_ctx.n
        dev = grad_a.device if grad_a is not None else grad_du.device
        ga = grad_a if grad_a is not None else torch.zeros(n, 3, dtype=torch.float32, device=dev)
        gd = grad_du if grad_du is not None else torch.zeros(n, dtype=torch.float32, device=dev)
        g4 = torch.cat([ga.float(), gd.float()[:, None]], 1).contiguous()
        gx, gv, gu = ctx.lib_ctx.force_backward(g4, h_mode=0)
        return gx[:, :3], gv[:, :3], gu, None, None, None


class SphForcesSolvedH(torch.autograd.Function):
    """(a, du/dt, h) = F(x, v, u) with h solved by the h iteration (Sec. 2.1.2), differentiable in x, v, u.

    ``forward(x, v, u, m, h0, lib_ctx)``: h0 (n,) is only the starting guess;
    ``lib_ctx`` a :class:`Context` with the h iteration (no FLAG_NO_H_ITER),
    whose h_tol sets how close h is to the root. Runs build_cells, density,
    force; h is returned as a non-differentiable output. The backward pass calls
    swift_gpu_force_backward with h_mode 1: h moves with x through the implicit
    function theorem. If the context ran other calls in between, backward
    first runs this forward's calls again from the saved inputs.
    """

    @staticmethod
    def forward(ctx, x, v, u, m, h0, lib_ctx):
        from . import _lib
        if lib_ctx.params.flags & _lib.FLAG_NO_H_ITER:
            raise ValueError("SphForcesSolvedH needs the h iteration (a context without FLAG_NO_H_ITER)")
        pos_h = torch.cat([x, h0[:, None]], 1).float().contiguous()
        vel_m = torch.cat([v, m[:, None]], 1).float().contiguous()
        uu = u.float().contiguous()
        d, out = SphForcesSolvedH._run(lib_ctx, pos_h, vel_m, uu)
        ctx.lib_ctx = lib_ctx
        ctx.calls = lib_ctx.calls
        ctx.inputs = (pos_h, vel_m, uu)
        ad = out["accel_dudt"]
        h = d["h"].clone()
        ctx.mark_non_differentiable(h)
        return ad[:, :3].clone(), ad[:, 3].clone(), h

    @staticmethod
    def _run(lib_ctx, pos_h, vel_m, uu):
        d = lib_ctx.density_checked(pos_h, vel_m)
        return d, lib_ctx.force(uu, want_dh=False, want_reductions=False)

    @staticmethod
    def backward(ctx, grad_a, grad_du, grad_h):
        if ctx.lib_ctx.calls != ctx.calls:  # the context moved on: restore this forward's state
            SphForcesSolvedH._run(ctx.lib_ctx, *ctx.inputs)
        n = ctx.lib_ctx.n
        dev = grad_a.device if grad_a is not None else grad_du.device
        ga = grad_a if grad_a is not None else torch.zeros(n, 3, dtype=torch.float32, device=dev)
        gd = grad_du if grad_du is not None else torch.zeros(n, dtype=torch.float32, device=dev)
        g4 = torch.cat([ga.float(), gd.float()[:, None]], 1).contiguous()
        gx, gv, gu = ctx.lib_ctx.force_backward(g4, h_mode=1)
        return gx[:, :3], gv[:, :3], gu, None, None, None


class StepGraph:
    """One hot-path step (build_cells, density, gradient + force) captured once in a CUDA graph.

    All inputs and outputs are fixed device tensors (``pos_h``, ``vel_m``, ``u``
    are read at every replay, so the caller refreshes them in place). The
    calls are made once outside capture first (the first call of each loop sets
    kernel attributes), then captured on a side stream; ``replay()`` re-issues
    the whole step with one launch from the host. The cell width is fixed at
    capture (``min_cell_width``; 0 lets the device choose it at every replay
    from the current h, as the direct calls do).
    """

    def __init__(self, ctx: Context, pos_h, vel_m, u, min_cell_width: float = 0.0, alpha_v=None, alpha_c=None,
                 fused: bool = True, active=None, rho4=None, curl_div=None):
        """``active`` (optional, uint8): only those particles are recomputed; ``rho4`` and ``curl_div`` then
        give the inactive particles' values (copied into the step's own output arrays, where the inactive
        entries stay from replay to replay)."""
        n = pos_h.shape[0]
        dev = pos_h.device
        self.ctx = ctx
        if active is not None and (rho4 is None or curl_div is None):
            raise ValueError("with an active subset, rho4 and curl_div carry the inactive particles' values")
        self.out = dict(h=torch.empty(n, dtype=_F32, device=dev),
                        rho4=rho4.clone() if rho4 is not None else torch.empty(n, 4, dtype=_F32, device=dev),
                        curl_div=curl_div.clone() if curl_div is not None else torch.empty(n, 4, dtype=_F32,
                                                                                          device=dev),
                        ngb=torch.zeros(n, dtype=torch.int32, device=dev),
                        vsig_lapu=torch.empty(n, 2, dtype=_F32, device=dev),
                        accel_dudt=torch.empty(n, 4, dtype=_F32, device=dev), dh_dt=torch.empty(n, dtype=_F32, device=dev),
                        reductions=torch.zeros(8, dtype=torch.float64, device=dev))
        o = self.out

        def body():
            ctx.build_cells(pos_h, min_cell_width)
            ctx.density(pos_h, vel_m, active, h_out=o["h"], rho4=o["rho4"], curl_div=o["curl_div"],
                        ngb_count=o["ngb"])
            if fused:
                ctx.gradient_force(u, alpha_v, alpha_c, vsig_lapu=o["vsig_lapu"], accel_dudt=o["accel_dudt"],
                                   dh_dt=o["dh_dt"], reductions=o["reductions"])
            else:
                ctx.gradient(u, vsig_lapu=o["vsig_lapu"])
                ctx.force(u, alpha_v, alpha_c, accel_dudt=o["accel_dudt"], dh_dt=o["dh_dt"],
                          reductions=o["reductions"])

        side = torch.cuda.Stream(device=dev)
        side.wait_stream(torch.cuda.current_stream(dev))
        with torch.cuda.stream(side):
            body()
        torch.cuda.current_stream(dev).wait_stream(side)
        torch.cuda.synchronize(dev)
        l0 = ctx.info()["launches"]
        self.graph = torch.cuda.CUDAGraph()
        with torch.cuda.graph(self.graph):
            body()
        self.launches_per_step = ctx.info()["launches"] - l0

    def replay(self):
        self.ctx.calls += 1  # the replayed calls replace the context's state like direct ones
        self.graph.replay()
        return self.out
