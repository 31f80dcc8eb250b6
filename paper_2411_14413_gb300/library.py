"""Materials-library analysis of simulated composition maps.

The paper compares the composition range that a simulated library covers with
the measured one and traces a smaller measured range to a cathode tilt that
differs from the assumed one (Sec. "Results", the ternary Pd-Pt-Ru library):
an increased common tilt shrinks the covered compositional area, so the tilt
can be estimated by simulating the library at several tilts and matching the
area (and the maps themselves) to the measurement.

* ``composition_maps`` runs a scene whose instances form consecutive libraries
  (e.g. ``workloads.scene_tilt_scan``: tilt-major, n_el instances per tilt) in
  ONE transport launch and converts every library's counts to an at.% map with
  the composition kernel (``sput_composition``).
* ``compositional_area`` is the share of the composition simplex covered by the
  convex hull of a map's points (the area of a ternary library in the ternary
  diagram; a volume share for four elements).
* ``diagnose_tilt`` estimates the common tilt of a measured map from maps
  simulated at a range of tilts, by the area criterion and by least squares
  with a fitted reference per simulated map (``fit_tilt``).
* ``fit_tilt_newton`` refines the tilt by Newton steps on the fitted-reference
  loss.  Its slope comes from the composition stage's adjoint
  (``sput_composition_backward``: dL/dcomposition -> dL/dcounts) contracted
  with the count derivative in tilt, a central difference of common random
  numbers across the tilt instances (t - h, t, t + h) of one batched launch
  (``TiltAdjoint``).  The tilt moves surfaces (the launch support itself), so
  the transport's likelihood-ratio score does not give that count derivative.
"""

from __future__ import annotations

import ctypes as C
import math

import numpy as np

from . import _native as N


def composition_maps(transport, n_el, patch_of_cell, ref_point, calibration, power, seed=None, stream=None):
    """[n_lib][n_points][n_el] at.% maps (device tensor) of the consecutive
    libraries of n_el instances in `transport`'s scene, from one run.

    calibration: host [n_el][6] rate-line rows (P_a, R_a, P_b, R_b, density, mass)
    shared by every library; power: host [n_el] in W."""
    return _composition_maps(transport, n_el, patch_of_cell, ref_point, calibration, power, seed, stream)[0]


def _composition_maps(transport, n_el, patch_of_cell, ref_point, calibration, power, seed, stream):
    """composition_maps, also returning the forward's patch counts [n_lib][n_el][n_points]
    and the device patch map (both needed by the composition backward)."""
    import torch

    L = transport.layout
    if L.n_instances % n_el:
        raise ValueError("the instance count is not a multiple of the library size")
    n_lib = L.n_instances // n_el
    dev = torch.device("cuda", transport.device)
    s = stream if stream is not None else torch.cuda.current_stream(transport.device).cuda_stream
    transport.run(seed=seed, stream=s, want_stats=False)
    counts = transport.t["counts"]
    if counts.dtype != torch.int64:
        raise ValueError("composition maps need int64 counts")
    n_cells = L.nx * L.ny
    patch = torch.as_tensor(np.ascontiguousarray(patch_of_cell, np.int32), device=dev)
    n_points = int(np.max(patch_of_cell)) + 1
    cal = np.ascontiguousarray(calibration, dtype=np.float64).reshape(n_el, 6)
    pw = np.ascontiguousarray(power, dtype=np.float64).reshape(n_el)
    patch_counts = torch.empty((n_lib, n_el, n_points), dtype=torch.float64, device=dev)
    comp = torch.empty((n_lib, n_points, n_el), dtype=torch.float64, device=dev)
    lib = N.load()
    for t in range(n_lib):
        rc = lib.sput_composition(n_el, n_cells, n_points,
                                  C.c_void_p(counts.data_ptr() + t * n_el * n_cells * counts.element_size()),
                                  C.c_void_p(patch.data_ptr()), int(ref_point), cal.ctypes.data_as(C.c_void_p),
                                  pw.ctypes.data_as(C.c_void_p), C.c_void_p(patch_counts[t].data_ptr()),
                                  C.c_void_p(comp[t].data_ptr()), C.c_void_p(s))
        N.check(rc, "sput_composition")
    return comp, patch_counts, patch


def compositional_area(comp):
    """Share of the composition simplex covered by the convex hull of the points.

    comp: [n_points][n_el] at.% (rows sum to 100), n_el = 3 or 4.  The points
    are mapped to the first n_el - 1 atomic fractions, an affine image of the
    simplex of volume 1/(n_el - 1)!, so the share is hull volume * (n_el - 1)!."""
    from scipy.spatial import ConvexHull

    x = np.asarray(comp, dtype=np.float64)
    n_el = x.shape[1]
    if n_el not in (3, 4):
        raise ValueError("compositional area is defined here for ternary and quaternary libraries")
    y = x[:, : n_el - 1] / 100.0
    return float(ConvexHull(y).volume * math.factorial(n_el - 1))


def _parabola_min(x, y):
    """Abscissa of the minimum of the parabola through the smallest sample and
    its two neighbours (the end sample itself at an end of the range)."""
    i = int(np.argmin(y))
    if i == 0 or i == len(x) - 1:
        return float(x[i])
    x0, x1, x2 = x[i - 1], x[i], x[i + 1]
    y0, y1, y2 = y[i - 1], y[i], y[i + 1]
    den = (x0 - x1) * (x0 - x2) * (x1 - x2)
    a = (x2 * (y1 - y0) + x1 * (y0 - y2) + x0 * (y2 - y1)) / den
    b = (x2 * x2 * (y0 - y1) + x1 * x1 * (y2 - y0) + x0 * x0 * (y1 - y2)) / den
    return float(-b / (2 * a)) if a > 0 else float(x1)


def _rescale(comp, log_k):
    """Composition map with element j's arrivals scaled by exp(log_k[j]) (the effect of
    another reference-patch count): c_j -> k_j c_j / sum_i k_i c_i, in at.%."""
    a = np.asarray(comp, dtype=np.float64) * np.exp(np.asarray(log_k))[None, :]
    return 100.0 * a / a.sum(axis=1, keepdims=True)


def fit_reference(sim, measured):
    """Per-element scale factors (element 0's fixed) of a simulated map that minimise its
    mean squared at.% difference to the measured map, and that difference.  The factors
    stand for the reference patch's counts, which every composition is normalised to and
    whose count noise rescales each element's whole map."""
    from scipy.optimize import least_squares

    sim = np.asarray(sim, dtype=np.float64)
    meas = np.asarray(measured, dtype=np.float64)
    n_el = meas.shape[1]

    def resid(x):
        return (_rescale(sim, np.concatenate([[0.0], x])) - meas).ravel()

    r = least_squares(resid, np.zeros(n_el - 1), x_scale=0.01, xtol=1e-12, ftol=1e-14)
    return np.exp(np.concatenate([[0.0], r.x])), float(np.mean(r.fun ** 2))


def fit_tilt(measured, tilts, simulated):
    """Least-squares tilt of a measured map with a fitted reference.

    Every simulated map gets its own reference factors (``fit_reference``), so neither the
    measured map's nor the simulated maps' reference-patch noise moves the estimate; the
    tilt is the minimum of the quadratic fitted, over all scanned tilts, to these
    mean squared differences (the scan's best tilt when the fit is not convex).
    Returns (tilt, the factors at the scanned tilt nearest to it, the per-tilt
    mean squared differences)."""
    tilts = np.asarray(tilts, dtype=np.float64)
    fits = [fit_reference(s, measured) for s in simulated]
    mse = np.array([f[1] for f in fits])
    c = np.polyfit(tilts, mse, 2)
    t = float(-c[1] / (2.0 * c[0])) if c[0] > 0 else float(tilts[int(np.argmin(mse))])
    t = float(np.clip(t, tilts[0], tilts[-1]))
    return t, fits[int(np.argmin(np.abs(tilts - t)))][0], mse


def diagnose_tilt(measured, tilts, simulated):
    """Common cathode tilt of a measured library map.

    measured: [n_points][n_el] at.%; simulated: [n_tilts][n_points][n_el] at.%
    at the increasing `tilts` (degrees).  Returns the tilt at which the
    simulated compositional area equals the measured one (linear interpolation
    between the bracketing tilts; None when no bracket exists; the criterion
    the paper uses), the least-squares tilt with a fitted reference
    (``fit_tilt``), the tilt of least mean squared difference of the maps as
    they are (parabola through the best three, which the reference patch's
    count noise shifts), and the per-tilt areas and mean squared differences."""
    tilts = np.asarray(tilts, dtype=np.float64)
    sim = np.asarray(simulated, dtype=np.float64)
    meas = np.asarray(measured, dtype=np.float64)
    areas = np.array([compositional_area(m) for m in sim])
    a_meas = compositional_area(meas)
    mse = ((sim - meas[None]) ** 2).mean(axis=(1, 2))
    t_area = None
    for i in range(len(tilts) - 1):
        a0, a1 = areas[i] - a_meas, areas[i + 1] - a_meas
        if a0 == 0.0:
            t_area = float(tilts[i])
            break
        if a0 * a1 < 0.0:
            t_area = float(tilts[i] + (tilts[i + 1] - tilts[i]) * a0 / (a0 - a1))
            break
    if t_area is None and areas[-1] == a_meas:
        t_area = float(tilts[-1])
    t_fit, factors, mse_fit = fit_tilt(meas, tilts, sim)
    return {"tilt_area": t_area, "tilt_lsq": t_fit, "lsq_factors": factors.tolist(), "lsq_mse": mse_fit.tolist(),
            "tilt_lsq_raw": _parabola_min(tilts, mse), "area_measured": a_meas, "areas": areas.tolist(),
            "mse": mse.tolist()}


def fitted_loss_grad(sim, measured):
    """Fitted-reference loss of a simulated map and its gradient in the map.

    L(sim) = min_k mean((R(sim, k) - measured)^2) with R the per-element rescale
    (``fit_reference``).  At the optimal factors k* the derivative of the minimum
    is the partial derivative at fixed k* (the factors are stationary there):
    with a = sim k*, S = sum_j a_j, R_j = 100 a_j / S and g = dL/dR,
    dL/dsim_l = (k*_l / S) (100 g_l - sum_j g_j R_j), row by row.
    Returns (L, k*, dL/dsim as [n_points][n_el])."""
    sim = np.asarray(sim, dtype=np.float64)
    meas = np.asarray(measured, dtype=np.float64)
    k, loss = fit_reference(sim, meas)
    a = sim * k[None, :]
    S = a.sum(axis=1, keepdims=True)
    R = 100.0 * a / S
    g = 2.0 * (R - meas) / R.size
    grad = (k[None, :] / S) * (100.0 * g - (g * R).sum(axis=1, keepdims=True))
    return loss, k, grad


class TiltAdjoint:
    """Fitted-reference loss of a measured map at a common tilt t, with its slope and
    curvature in t, from ONE batched launch of the library at tilts (t - h, t, t + h).

    make_scene(tilts) must return a tilt-major scene of n_el instances per tilt in
    which every tilt's instance of an element draws the same random stream (common
    random numbers, e.g. ``workloads.scene_tilt_scan(..., common_random_numbers=True)``).
    evaluate(t, h) returns
      loss:  the fitted-reference loss at t (``fitted_loss_grad``);
      slope: dL/dt, the adjoint of the composition stage at t (dL/dcomposition
             -> dL/dcounts, ``sput_composition_backward``) contracted with the
             central difference of the counts, (counts(t + h) - counts(t - h)) / 2h;
      curv:  (L(t + h) - 2 L(t) + L(t - h)) / h^2 from the three fitted losses;
      factors: the reference factors at t."""

    def __init__(self, make_scene, measured, patch_of_cell, ref_point, calibration, power, seed=0, device=0):
        self.make_scene = make_scene
        self.measured = np.asarray(measured, dtype=np.float64)
        self.patch_of_cell = np.ascontiguousarray(patch_of_cell, np.int32)
        self.ref = int(ref_point)
        self.n_el = self.measured.shape[1]
        self.cal = np.ascontiguousarray(calibration, dtype=np.float64).reshape(self.n_el, 6)
        self.power = np.ascontiguousarray(power, dtype=np.float64).reshape(self.n_el)
        self.seed = seed
        self.device = device
        self.launches = 0

    def evaluate(self, t, h):
        import torch

        from . import api

        sc = self.make_scene([t - h, t, t + h])
        if len(sc.instances) != 3 * self.n_el:
            raise ValueError("the scene must hold n_el instances at each of the three tilts")
        tr = api.Transport(sc, device=self.device, energy=False, prim_counts=False)
        try:
            s = torch.cuda.current_stream(self.device).cuda_stream
            comp, patch_counts, patch = _composition_maps(tr, self.n_el, self.patch_of_cell, self.ref, self.cal,
                                                          self.power, self.seed, s)
            self.launches += 1
            comp_h = comp.cpu().numpy()
            L_m = fit_reference(comp_h[0], self.measured)[1]
            L_p = fit_reference(comp_h[2], self.measured)[1]
            loss, k, grad = fitted_loss_grad(comp_h[1], self.measured)
            dev = comp.device
            n_cells = tr.layout.nx * tr.layout.ny
            n_points = comp.shape[1]
            g_comp = torch.as_tensor(np.ascontiguousarray(grad), dtype=torch.float64, device=dev)
            g_patch = torch.empty((self.n_el, n_points), dtype=torch.float64, device=dev)
            g_counts = torch.empty((self.n_el, n_cells), dtype=torch.float64, device=dev)
            g_power = torch.empty(self.n_el, dtype=torch.float64, device=dev)
            rc = N.load().sput_composition_backward(
                self.n_el, n_cells, n_points, C.c_void_p(patch_counts[1].data_ptr()), C.c_void_p(patch.data_ptr()),
                self.ref, self.cal.ctypes.data_as(C.c_void_p), self.power.ctypes.data_as(C.c_void_p),
                C.c_void_p(g_comp.data_ptr()), C.c_void_p(g_patch.data_ptr()), C.c_void_p(g_counts.data_ptr()),
                C.c_void_p(g_power.data_ptr()), C.c_void_p(s))
            N.check(rc, "sput_composition_backward")
            counts = tr.t["counts"].reshape(3, self.n_el, n_cells)
            dcounts = (counts[2] - counts[0]).to(torch.float64) / (2.0 * h)
            slope = float((g_counts * dcounts).sum().cpu())
        finally:
            tr.close()
        return {"t": float(t), "loss": loss, "slope": slope, "curv": (L_p - 2.0 * loss + L_m) / (h * h),
                "losses": [L_m, loss, L_p], "factors": k.tolist()}


def fit_tilt_newton(evaluate, t0, h=1.0, iters=8, tol=0.02, bounds=(0.0, 60.0)):
    """Safeguarded Newton iteration on the tilt.

    evaluate(t, h) gives the loss, its slope and curvature at t (``TiltAdjoint.evaluate``).
    The Newton step -slope/curv is clipped to +-h (a step of h downhill where the
    curvature is not positive).  Once the slope has changed sign between two evaluated
    tilts, they bracket the minimum: a step that leaves the bracket bisects it instead,
    and the iteration ends when the bracket is narrower than tol (the slope of a finite
    sample is jagged on small scales, so a bare Newton iteration can cycle there).  It
    also ends when a step is shorter than tol.  Returns (tilt, the evaluations in order)."""
    t = float(t0)
    lo, hi = -math.inf, math.inf
    hist = []
    for _ in range(iters):
        r = evaluate(t, h)
        hist.append(r)
        if r["slope"] > 0.0:
            hi = min(hi, t)
        else:
            lo = max(lo, t)
        step = -r["slope"] / r["curv"] if r["curv"] > 0.0 else -math.copysign(h, r["slope"])
        t_new = t + float(np.clip(step, -h, h))
        if math.isfinite(lo) and math.isfinite(hi):
            if hi - lo < tol:
                t_new = 0.5 * (lo + hi)
                r["step"] = t_new - t
                t = t_new
                break
            if not lo < t_new < hi:
                t_new = 0.5 * (lo + hi)
        t_new = float(np.clip(t_new, *bounds))
        r["step"] = t_new - t
        t = t_new
        if abs(r["step"]) < tol:
            break
    return t, hist
