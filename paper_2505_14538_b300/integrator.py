"""Kick-drift-kick leapfrog of the SPH system on the library's kernels.

One step (swift_gpu_time.h): kick + drift, cells + density (h iteration) at
the drifted positions and predicted velocities, viscosity switch (Eqs.
12-15), gradient + force with the predicted u and the new alpha_v, second
half kick with the alpha_c update (Eqs. 21, 23, 24) and the next step size.
Every stage is a library call; this class owns the device buffers and the
device clock, and can capture whole steps in a CUDA graph.
"""
from __future__ import annotations

import torch

from . import _lib
from .sph import Context, SwiftGPUError, make_time_params, new_clock, read_clock

_F32 = torch.float32


class Integrator:
    """State of a leapfrog integration (all n particles, one global step).

    ``pos_h``, ``vel_m``, ``u`` (CUDA float32, (n, 4), (n, 4), (n,)) are
    advanced in place. ``alpha_v`` / ``alpha_c`` default to the context's
    constants and then evolve per particle. ``t_end`` > 0 stops the clock
    there (later steps have dt = 0). Keyword arguments set
    swift_gpu_time_params fields (cfl, dt_max, alpha_v_max, ...).
    """

    def __init__(self, ctx: Context, pos_h, vel_m, u, alpha_v=None, alpha_c=None, t_end: float = 0.0,
                 min_cell_width: float = 0.0, **time_params):
        n = pos_h.shape[0]
        dev = pos_h.device
        self.ctx, self.n = ctx, n
        self.tp = make_time_params(**time_params)
        self.pos_h, self.vel_m, self.u = pos_h, vel_m, u
        self.alpha_v = alpha_v if alpha_v is not None else torch.full((n,), float(ctx.params.alpha_v), device=dev)
        self.alpha_c = alpha_c if alpha_c is not None else torch.full((n,), float(ctx.params.alpha_c), device=dev)
        self.min_cell_width = float(min_cell_width)
        e = lambda *shape: torch.zeros(*shape, dtype=_F32, device=dev)
        self.vel_pred, self.u_pred = e(n, 4), e(n)
        self.h, self.rho4, self.curl_div = e(n), e(n, 4), e(n, 4)
        self.ngb = torch.zeros(n, dtype=torch.int32, device=dev)
        self.vsig_lapu, self.accel_dudt, self.dh_dt, self.div_prev = e(n, 2), e(n, 4), e(n), e(n)
        self.reductions = torch.zeros(8, dtype=torch.float64, device=dev)
        self.clock = new_clock(t_end, dev)
        self.primed = False

    # --------------------------------------------------------------- stages
    def _loops(self, vel, u, check):
        c = self.ctx
        c.density_checked(self.pos_h, vel, None, self.rho4, self.curl_div, self.min_cell_width, check,
                          h_out=self.h, ngb_count=self.ngb)
        c.viscosity_switch(self.tp, self.clock, self.h, u, self.curl_div, self.vsig_lapu, self.div_prev,
                           self.alpha_v)
        c.gradient_force(u, self.alpha_v, self.alpha_c, vsig_lapu=self.vsig_lapu, accel_dudt=self.accel_dudt,
                         dh_dt=self.dh_dt, reductions=self.reductions)

    def prime(self, check: bool = True):
        """Loops at the initial state (clock dt = 0): rates, v_sig, div v and the first step size."""
        self._loops(self.vel_m, self.u, check)
        self.ctx.kick_finish(self.tp, self.clock, self.h, self.pos_h, self.vel_m, self.u, self.accel_dudt,
                             self.vsig_lapu, self.alpha_v, self.alpha_c)
        self.primed = True

    def step(self, check: bool = True):
        """One leapfrog step. check=True reads the density status (one host synchronisation)."""
        if not self.primed:
            raise RuntimeError("Integrator.prime() must run before the first step")
        c = self.ctx
        c.kick_drift(self.tp, self.clock, self.pos_h, self.vel_m, self.u, self.accel_dudt, self.dh_dt,
                     self.vel_pred, self.u_pred)
        self._loops(self.vel_pred, self.u_pred, check)
        c.kick_finish(self.tp, self.clock, self.h, self.pos_h, self.vel_m, self.u, self.accel_dudt,
                      self.vsig_lapu, self.alpha_v, self.alpha_c)

    def clock_state(self) -> dict:
        return read_clock(self.clock)

    def run_until(self, t_end: float, max_steps: int = 100000, check: bool = True) -> dict:
        """Step until the clock reaches t_end (which must be the clock's own t_end, or it is set to it)."""
        st = self.clock_state()
        if st["t_end"] != t_end:
            raw = _lib.Clock(st["t"], float(t_end), st["dt"], st["dt_next"], st["step"])
            self.clock.copy_(torch.frombuffer(bytearray(bytes(raw)), dtype=torch.float64))
        for _ in range(max_steps):
            if self.clock_state()["t"] >= t_end:
                break
            self.step(check)
        return self.clock_state()

    def capture(self, steps: int = 1) -> "torch.cuda.CUDAGraph":
        """Capture `steps` steps (without status checks) in one CUDA graph; replay() advances them.

        Cell widths are chosen on the device at every replay from the current
        h (min_cell_width 0) unless a fixed width was given. Read the status
        with ctx.sync_status() after replays.
        """
        if not self.primed:
            raise RuntimeError("Integrator.prime() must run before capture")
        graph = torch.cuda.CUDAGraph()
        dev = self.pos_h.device
        side = torch.cuda.Stream(device=dev)
        side.wait_stream(torch.cuda.current_stream(dev))
        torch.cuda.synchronize(dev)
        with torch.cuda.graph(graph, stream=side):
            for _ in range(steps):
                self.step(check=False)
        return graph

    def check_status(self):
        code, detail = self.ctx.sync_status()
        if code not in (_lib.OK, _lib.ERR_H_NOT_CONVERGED):
            raise SwiftGPUError(code, "integration step", detail)
        return code, detail
