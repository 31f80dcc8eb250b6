"""Composition-map gradients with respect to gas pressure and cathode powers.

``CompositionMap`` is a torch.autograd.Function over the library's kernels:
forward = transport with score tallies (sput_run) followed by the
counts -> at.% map (sput_composition); backward = the composition map's
backward pass (sput_composition_backward, which also gives dL/dP through the
rate lines) followed by the likelihood-ratio contraction for the pressure
(sput_backward) and, with voltage lines, the power's path through the
discharge voltage to the Thompson cut-off (sput_voltage_backward).  Python
only marshals pointers.

``inverse_solve`` fits (ln p, P_1..P_n) to a target composition map with
Adam, using common random numbers (a fixed seed) in every step.
"""

from __future__ import annotations

import ctypes as C
import math

import numpy as np

from . import _native as N
from . import api


def _ptr(t):
    return C.c_void_p(t.data_ptr())


class MapSetup:
    """Transport scene + measurement patches + calibration for one composition map.

    voltage (optional, host [n_cath][4] = P_a, V_a, P_b, V_b): the discharge
    voltage of each cathode as the line through two (power, voltage) points
    (Table S1); the incident ion energy E_i (eV, singly charged ions) then
    follows the power, which moves the Thompson cut-off E_max = k Lambda E_i - U_s,
    and backward() adds that path to dL/dP (boundary run + sput_voltage_backward).
    The voltage arithmetic itself runs in the library (sput_ion_energy and
    sput_voltage_backward); this class only marshals."""

    def __init__(self, scene, patch_of_cell, ref_point, calibration, device=0, voltage=None):
        import torch

        self.scene = scene
        self.device = device
        self.tr = api.Transport(scene, device=device, score=True, energy=False, prim_counts=True)
        L = self.tr.layout
        self.n_cath = L.n_instances
        self.n_cells = L.nx * L.ny
        self.n_points = int(np.max(patch_of_cell)) + 1
        self.ref = int(ref_point)
        dev = torch.device("cuda", device)
        self.patch = torch.as_tensor(np.ascontiguousarray(patch_of_cell, np.int32), device=dev)
        self.cal = np.ascontiguousarray(calibration, dtype=np.float64).reshape(self.n_cath, 6)
        self.patch_counts = torch.zeros((self.n_cath, self.n_points), dtype=torch.float64, device=dev)
        self.grad_patch = torch.zeros_like(self.patch_counts)
        self.grad_counts = torch.zeros((self.n_cath, self.n_cells), dtype=torch.float64, device=dev)
        self.grad_logp = torch.zeros(self.n_cath, dtype=torch.float64, device=dev)
        self.grad_power = torch.zeros(self.n_cath, dtype=torch.float64, device=dev)
        self.comp = torch.zeros((self.n_points, self.n_cath), dtype=torch.float64, device=dev)
        self.volt = None if voltage is None else np.ascontiguousarray(voltage, dtype=np.float64).reshape(self.n_cath, 4)
        self.seed = None
        if self.volt is not None:
            self.counts_cut = torch.zeros_like(self.tr.t["counts"])
            self._cut_tal = N.sput_tallies()
            self._cut_tal.counts = self.counts_cut.data_ptr()
            self.grad_Ei = torch.zeros(self.n_cath, dtype=torch.float64, device=dev)

    def stream(self):
        import torch

        return torch.cuda.current_stream(self.device).cuda_stream

    def ion_energy(self, power):
        """E_i (eV) of every cathode at the given powers, from the voltage lines (sput_ion_energy)."""
        pw = np.ascontiguousarray(power, dtype=np.float64)
        out = np.empty(self.n_cath, dtype=np.float64)
        rc = N.load().sput_ion_energy(self.n_cath, self.volt.ctypes.data_as(C.c_void_p), pw.ctypes.data_as(C.c_void_p),
                                      out.ctypes.data_as(C.c_void_p))
        N.check(rc, "sput_ion_energy")
        return out

    def set_conditions(self, p, power=None):
        sc = self.scene.with_pressure(float(p))
        if self.volt is not None and power is not None:
            sc = sc.with_ion_energy(self.ion_energy(power))
        self.scene = sc
        self.tr.set_instances(sc)

    def set_pressure(self, p):
        self.set_conditions(p)

    def forward(self, p, power, seed):
        """composition[n_points][n_cath] (at.%) for pressure p and powers (host array)."""
        self.set_conditions(p, power)
        self.seed = seed
        self.tr.run(seed=seed, want_stats=False)
        pw = np.ascontiguousarray(power, dtype=np.float64)
        rc = N.load().sput_composition(self.n_cath, self.n_cells, self.n_points, _ptr(self.tr.t["counts"]),
                                       _ptr(self.patch), self.ref, self.cal.ctypes.data_as(C.c_void_p),
                                       pw.ctypes.data_as(C.c_void_p), _ptr(self.patch_counts), _ptr(self.comp),
                                       C.c_void_p(self.stream()))
        N.check(rc, "sput_composition")
        return self.comp

    def backward(self, grad_comp, power):
        """(dL/d ln p per instance, dL/dP per cathode) from dL/dcomposition."""
        pw = np.ascontiguousarray(power, dtype=np.float64)
        g = grad_comp.contiguous()
        L = N.load()
        rc = L.sput_composition_backward(self.n_cath, self.n_cells, self.n_points, _ptr(self.patch_counts),
                                         _ptr(self.patch), self.ref, self.cal.ctypes.data_as(C.c_void_p),
                                         pw.ctypes.data_as(C.c_void_p), _ptr(g), _ptr(self.grad_patch),
                                         _ptr(self.grad_counts), _ptr(self.grad_power), C.c_void_p(self.stream()))
        N.check(rc, "sput_composition_backward")
        rc = L.sput_backward(self.tr.h, _ptr(self.grad_counts), _ptr(self.tr.t["score"]), _ptr(self.grad_logp),
                             C.c_void_p(self.stream()))
        N.check(rc, "sput_backward")
        if self.volt is not None:
            # the same particles launched at E_max: the moving end of the Thompson support
            o = api.run_opts(seed=self.seed, flags=N.SPUT_RUN_LAUNCH_AT_CUTOFF)
            api.sput_run(self.tr.h, o, self.stream(), self._cut_tal, False)
            # dL/dE_i, and dL/dE_i dE_i/dP added to the rate-line term of dL/dP
            rc = L.sput_voltage_backward(self.tr.h, self.volt.ctypes.data_as(C.c_void_p), _ptr(self.grad_counts),
                                         _ptr(self.tr.t["counts"]), _ptr(self.counts_cut), _ptr(self.grad_Ei),
                                         _ptr(self.grad_power), C.c_void_p(self.stream()))
            N.check(rc, "sput_voltage_backward")
        return self.grad_logp, self.grad_power

    def close(self):
        self.tr.close()


def composition_function():
    import torch

    class CompositionMap(torch.autograd.Function):
        """composition = CompositionMap.apply(log_p, power, setup, seed); log_p is shared by all cathodes."""

        @staticmethod
        def forward(ctx, log_p, power, setup, seed):
            p = math.exp(float(log_p.detach().cpu()))
            pw = power.detach().cpu().numpy().astype(np.float64)
            comp = setup.forward(p, pw, seed).clone()
            ctx.setup = setup
            ctx.power = pw
            return comp

        @staticmethod
        def backward(ctx, grad_comp):
            glogp, gpow = ctx.setup.backward(grad_comp.to(torch.float64), ctx.power)
            return glogp.sum().reshape(()).to(torch.float64), gpow.clone(), None, None

    return CompositionMap


def inverse_solve(setup, target, log_p0, power0, steps=50, lr=0.1, seed=0, power_bounds=(2.0, 80.0),
                  log_p_bounds=(math.log(0.05), math.log(5.0)), history=None, lr_final=0.1):
    """Adam on (ln p, ln P) minimising the mean squared composition error (at.%^2),
    learning rate decaying along a cosine from lr to lr * lr_final.  The map
    depends mostly on rate ratios, so a common scaling of all powers is only
    weakly determined (through the rate lines' intercepts)."""
    import torch

    dev = target.device
    CompositionMap = composition_function()
    log_p = torch.tensor(float(log_p0), dtype=torch.float64, device=dev, requires_grad=True)
    # powers are optimised in log space so that one learning rate suits all cathodes
    log_pw = torch.tensor(np.log(np.asarray(power0, float)), dtype=torch.float64, device=dev, requires_grad=True)
    opt = torch.optim.Adam([log_p, log_pw], lr=lr)
    out = []
    for it in range(steps):
        for g in opt.param_groups:
            g["lr"] = lr * (lr_final + (1 - lr_final) * 0.5 * (1 + math.cos(math.pi * it / max(1, steps - 1))))
        opt.zero_grad()
        comp = CompositionMap.apply(log_p, torch.exp(log_pw), setup, seed)
        loss = ((comp - target) ** 2).mean()
        loss.backward()
        opt.step()
        with torch.no_grad():
            log_p.clamp_(*log_p_bounds)
            log_pw.clamp_(math.log(power_bounds[0]), math.log(power_bounds[1]))
        out.append({"step": it, "loss": float(loss.detach()), "p": float(torch.exp(log_p).detach()),
                    "power": torch.exp(log_pw).detach().cpu().numpy().tolist()})
        if history is not None:
            history.append(out[-1])
    return out
