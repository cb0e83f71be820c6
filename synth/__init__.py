"""Seeded synthetic inputs for the HWFV1 workloads.

This module is shared by the oracle tests and by the CUDA path's tests and
benchmark.  It only builds problem descriptions (plain dicts) and initial
fields (numpy arrays, row-major ``[j, i]`` over the finest 2^L x 2^L grid, j
growing with y); it holds none of the method's arithmetic.

Workloads (the paper's test cases, Sec. 3, replaced by seeded stand-ins):

* ``circular_dam_break`` -- the circular 2D dam-break of Sec. 3.2 rescaled to
  the unit square.
* ``bumpy_dam_break`` -- a dam-break over seeded Gaussian humps with wet/dry
  fronts, standing in for the hump tests of Sec. 3.1.
* ``terrain_flood`` -- a seeded 1/f^2 spectral DEM with a carved channel and
  an inflow hydrograph, standing in for the DEM-based tests of Sec. 3.3;
  ``terrain_flood_peak`` is its state at the hydrograph peak with the channel
  running full.
* ``ensemble`` -- many independent bumpy dam-breaks of mixed depth L.
* small fixtures for the pins: lake at rest, a wet mound in a closed basin,
  pseudo-2D dam-break (Sec. 3.2),
  uniform frictional flow, a closed basin with inflow.
"""
from __future__ import annotations

import numpy as np

BC = {"closed": 0, "transmissive": 1, "inflow": 2}


def problem(L, lx=1.0, ly=1.0, x0=0.0, y0=0.0, eps=1e-3, cfl=0.5, g=9.80665,
            manning_n=0.0, tol_h=1e-3, dt_max=1.0, bc=("closed",) * 4,
            inflow=None, reg_predict=True, reg_close=True, flux_match=False):
    """Problem description: domain, maximum level L, threshold eps, CFL,
    gravity, Manning n, wet/dry tolerance, boundary kinds (W, E, S, N) and an
    optional inflow ``{"a0": first finest cell, "a1": end, "t": [...],
    "Q": [...]}`` on the side whose kind is ``"inflow"``; ``flux_match`` selects
    the conservative variant with matched fluxes at resolution changes."""
    bc = tuple(bc)
    assert len(bc) == 4 and all(b in BC for b in bc)
    assert sum(b == "inflow" for b in bc) <= 1
    return dict(L=int(L), lx=float(lx), ly=float(ly), x0=float(x0), y0=float(y0),
                eps=float(eps), cfl=float(cfl), g=float(g), manning_n=float(manning_n),
                tol_h=float(tol_h), dt_max=float(dt_max), bc=bc, inflow=inflow,
                reg_predict=bool(reg_predict), reg_close=bool(reg_close),
                flux_match=bool(flux_match))


def centres(p):
    """Cell-centre coordinates (x, y) of the finest grid, each [j, i]."""
    n = 1 << p["L"]
    dx, dy = p["lx"] / n, p["ly"] / n
    x = p["x0"] + (np.arange(n) + 0.5) * dx
    y = p["y0"] + (np.arange(n) + 0.5) * dy
    return np.meshgrid(x, y, indexing="xy")


def _fields(p, eta, z, qx=None, qy=None):
    h = np.maximum(0.0, eta - z)
    qx = np.zeros_like(h) if qx is None else qx
    qy = np.zeros_like(h) if qy is None else qy
    return dict(h=np.ascontiguousarray(h, dtype=np.float64),
                qx=np.ascontiguousarray(qx, dtype=np.float64),
                qy=np.ascontiguousarray(qy, dtype=np.float64),
                z=np.ascontiguousarray(z, dtype=np.float64))


def gaussian_humps(p, rng, count=8, amp=(0.1, 0.6), sigma=(0.02, 0.08)):
    """Sum of `count` Gaussian humps with heights U[amp], widths U[sigma] (as a
    fraction of the domain side) and centres U[domain]."""
    x, y = centres(p)
    z = np.zeros_like(x)
    for _ in range(count):
        a = rng.uniform(*amp)
        s = rng.uniform(*sigma) * p["lx"]
        cx = p["x0"] + rng.uniform(0.0, 1.0) * p["lx"]
        cy = p["y0"] + rng.uniform(0.0, 1.0) * p["ly"]
        z += a * np.exp(-((x - cx) ** 2 + (y - cy) ** 2) / (2.0 * s * s))
    return z


# --------------------------------------------------------------------------
# Workloads
# --------------------------------------------------------------------------

def circular_dam_break(L=6, eps=1e-3, radius=0.25, h_in=2.0, h_out=1.0):
    """Circular dam-break on the unit square (Sec. 3.2 rescaled): flat bed,
    depth h_in inside the circle of the given radius about the centre, h_out
    outside, at rest, transmissive sides, no friction."""
    p = problem(L, eps=eps, bc=("transmissive",) * 4)
    x, y = centres(p)
    r = np.sqrt((x - 0.5) ** 2 + (y - 0.5) ** 2)
    z = np.zeros_like(x)
    eta = np.where(r < radius, h_in, h_out)
    return p, _fields(p, eta, z)


def dry_bed_dam_break(L=8, eps=1e-3, x1=0.2, y1=0.3, h0=1.0, relief=0.0, seed=7):
    """A block of still water (free surface h0 over x < x1, y < y1) released
    onto dry ground (h = 0 elsewhere), closed walls, no friction.  The bed is
    flat, or with relief > 0 a seeded 1/f^2 surface of that relief (rough
    ground: its details keep the tree fine everywhere)."""
    p = problem(L, eps=eps, bc=("closed",) * 4)
    x, y = centres(p)
    z = np.zeros_like(x) if relief <= 0 else spectral_dem(1 << L, seed, relief)
    eta = np.where((x < x1) & (y < y1), h0, 0.0)
    return p, _fields(p, eta, z)


def columns_dam_break(L=8, eps=1e-3, seed=0, k=3, h_out=1.0):
    """k seeded circular water columns collapsing on a flat bed: centres
    U[0.2, 0.8]^2, radii U[0.05, 0.15], depths U[1.3, 2.0] over h_out, at rest,
    closed walls, no friction.  Only the moving flow sets the refinement
    (the bed has no details)."""
    p = problem(L, eps=eps, bc=("closed",) * 4)
    rng = np.random.default_rng(seed)
    x, y = centres(p)
    eta = np.full_like(x, h_out)
    for _ in range(k):
        cx, cy = rng.uniform(0.2, 0.8, size=2)
        r = rng.uniform(0.05, 0.15)
        hin = rng.uniform(1.3, 2.0)
        eta = np.where((x - cx) ** 2 + (y - cy) ** 2 < r * r, np.maximum(eta, hin), eta)
    return p, _fields(p, eta, np.zeros_like(x))


def bumpy_dam_break(L=10, eps=1e-3, seed=2, eta_up=1.0, eta_down=0.5, dam_x=0.3):
    """Dam-break over 8 seeded Gaussian humps on the unit square: free
    surface eta_up behind x = dam_x, eta_down elsewhere, closed walls; humps
    that reach above the water make wet/dry fronts."""
    p = problem(L, eps=eps, bc=("closed",) * 4)
    rng = np.random.default_rng(seed)
    z = gaussian_humps(p, rng)
    x, _ = centres(p)
    eta = np.where(x < dam_x, eta_up, eta_down)
    return p, _fields(p, eta, z)


def spectral_dem(n, seed, relief):
    """Seeded 1/f^2 spectral DEM on an n x n grid: real part of the inverse
    FFT of complex Gaussian noise times |f|^-2 (zero mean), scaled to the
    given relief (max - min) with minimum 0."""
    rng = np.random.default_rng(seed)
    fx = np.fft.fftfreq(n)
    f = np.sqrt(fx[None, :] ** 2 + fx[:, None] ** 2)
    f[0, 0] = np.inf
    noise = rng.standard_normal((n, n)) + 1j * rng.standard_normal((n, n))
    z = np.real(np.fft.ifft2(noise / f ** 2))
    z = (z - z.min()) / (z.max() - z.min()) * relief
    return z


def terrain_flood(L=12, eps=1e-3, seed=3, side_m=10_000.0, relief=50.0, width=60.0,
                  depth=4.0, tilt=1e-3, q_peak=500.0, t_peak=1800.0, t_end=3600.0,
                  manning_n=0.03, amplitude=None, wavelength=None, fill=0.0, fill_q=0.0):
    """Synthetic terrain flood: a seeded 1/f^2 DEM of the given relief over a
    square of side `side_m`, tilted down W->E by `tilt`, with a channel of the
    given width and depth carved along a sinusoidal W->E centreline.  The
    domain starts dry; a triangular hydrograph (0 -> q_peak at t_peak -> 0 at
    t_end, m^3/s) enters through the channel inlet on the west side, the
    other sides are closed walls; Manning friction n.  With fill > 0 the
    channel instead starts `fill` metres deep with discharge fill_q (m^2/s,
    towards +x) along its whole length: a wet state for one-step checks."""
    n = 1 << L
    amplitude = 0.1 * side_m if amplitude is None else amplitude
    wavelength = 0.5 * side_m if wavelength is None else wavelength
    p0 = problem(L, lx=side_m, ly=side_m)
    x, y = centres(p0)
    z = spectral_dem(n, seed, relief)
    z = z + tilt * (side_m - x)
    yc = 0.5 * side_m + amplitude * np.sin(2.0 * np.pi * x / wavelength)
    z = np.where(np.abs(y - yc) < 0.5 * width, z - depth, z)
    dy = side_m / n
    yc0 = 0.5 * side_m
    a0 = int(np.floor((yc0 - 0.5 * width) / dy))
    a1 = int(np.ceil((yc0 + 0.5 * width) / dy))
    inflow = dict(a0=a0, a1=a1, t=[0.0, t_peak, t_end], Q=[0.0, q_peak, 0.0])
    p = problem(L, lx=side_m, ly=side_m, eps=eps, manning_n=manning_n,
                bc=("inflow", "closed", "closed", "closed"), inflow=inflow)
    if fill > 0.0:
        inside = np.abs(y - yc) < 0.5 * width
        h = np.where(inside, fill, 0.0)
        return p, dict(h=np.ascontiguousarray(h), qx=np.ascontiguousarray(np.where(inside, fill_q, 0.0)),
                       qy=np.zeros_like(h), z=np.ascontiguousarray(z))
    eta = np.full_like(z, -1e9)          # dry start
    return p, _fields(p, eta, z)


def terrain_flood_peak(L=12, eps=1e-3, depth=3.45, q=8.33):
    """The terrain flood at its hydrograph peak, t = 1800 s: the channel runs
    `depth` metres deep (3.45 m is the Manning normal depth of the peak's
    500 m^3/s through the 60 m channel on the 0.1 % tilt) with `q` m^2/s
    towards +x, the rest of the domain dry.  Returns (problem, fields, t)."""
    p, f = terrain_flood(L=L, eps=eps, fill=depth, fill_q=q)
    return p, f, 1800.0


def ensemble(count=64, seed=4, levels=(7, 8, 9, 10), eps=1e-3):
    """Batched ensemble: `count` independent bumpy dam-breaks with L drawn
    uniformly from `levels`, hump seeds seed+d and upstream levels U[0.5, 2]."""
    rng = np.random.default_rng(seed)
    out = []
    for d in range(count):
        L = int(rng.choice(levels))
        eta_up = float(rng.uniform(0.5, 2.0))
        out.append(bumpy_dam_break(L=L, eps=eps, seed=seed + d, eta_up=eta_up))
    return out


# --------------------------------------------------------------------------
# Small fixtures for the pins
# --------------------------------------------------------------------------

def lake_at_rest(L=6, eps=1e-3, seed=5, eta=1.0, wet=True):
    """Still water over seeded humps, closed walls.  With wet=True the humps
    stay below the surface (fully wet); otherwise some emerge (Table 3's
    partly dry setting)."""
    p = problem(L, eps=eps, bc=("closed",) * 4)
    rng = np.random.default_rng(seed)
    amp = (0.1, 0.6) if wet else (0.6, 1.4)
    z = gaussian_humps(p, rng, amp=amp)
    return p, _fields(p, np.full_like(z, eta), z)


def wet_mound(L=6, eps=1e-3, seed=5, eta=1.0, mound=0.3):
    """A raised free-surface mound released over seeded humps in a closed
    basin, fully wet: the finest depths under a leaf hand its volume down
    unchanged, so the volume changes only through the fluxes."""
    p, f = lake_at_rest(L=L, eps=eps, seed=seed, eta=eta)
    x, y = centres(p)
    eta_m = eta + mound * np.exp(-((x - 0.3) ** 2 + (y - 0.6) ** 2) / 0.01)
    return p, _fields(p, eta_m, f["z"])


def pseudo_2d_dam_break(L=7, eps=0.0, h_up=6.0, h_down=2.0, dam_x=10.0):
    """Pseudo-2D dam-break of Sec. 3.2: 50 m x 25 m flat frictionless
    channel, open (transmissive) boundaries, dam at x = dam_x."""
    p = problem(L, lx=50.0, ly=25.0, eps=eps, bc=("transmissive",) * 4)
    x, _ = centres(p)
    z = np.zeros_like(x)
    eta = np.where(x < dam_x, h_up, h_down)
    return p, _fields(p, eta, z)


def ritter_dam_break(L=6, eps=0.0, h0=1.0, water="west", side_m=100.0):
    """Dam break onto a dry flat bed (Ritter's problem): still water h0 on
    one half of a square (``water`` = "west" or "east"), dry ground on the
    other, transmissive sides.  Mirror images of each other."""
    p = problem(L, lx=side_m, ly=side_m, eps=eps, bc=("transmissive",) * 4)
    x, _ = centres(p)
    wet = (x < 0.5 * side_m) if water == "west" else (x > 0.5 * side_m)
    return p, _fields(p, np.where(wet, h0, 0.0), np.zeros_like(x))


def uniform_flow(L=4, h=1.0, u=2.0, manning_n=0.03, eps=0.0):
    """Uniform depth and velocity on a flat bed with transmissive sides and
    Manning friction: the fluxes cancel and only friction acts."""
    p = problem(L, eps=eps, manning_n=manning_n, bc=("transmissive",) * 4)
    x, _ = centres(p)
    z = np.zeros_like(x)
    return p, _fields(p, np.full_like(x, h), z, qx=np.full_like(x, h * u))


def inflow_basin(L=5, eps=1e-3, q=2.0, seed=6):
    """Closed basin over humps with still water and a constant inflow Q
    through part of the west side."""
    n = 1 << L
    inflow = dict(a0=n // 4, a1=n // 2, t=[0.0, 1000.0], Q=[q, q])
    p = problem(L, eps=eps, bc=("inflow", "closed", "closed", "closed"), inflow=inflow)
    rng = np.random.default_rng(seed)
    z = gaussian_humps(p, rng, amp=(0.1, 0.3))
    return p, _fields(p, np.full_like(z, 0.5), z)


def random_state(L, seed, dyadic=False):
    """Random finest fields for encode/decode pins.  With dyadic=True every
    value is k * 2^-10 with |k| < 2^20, so all the sums of Eq. 3/4 are exact."""
    rng = np.random.default_rng(seed)
    n = 1 << L
    if dyadic:
        return rng.integers(-(1 << 20), 1 << 20, size=(n, n)).astype(np.float64) * 2.0 ** -10
    return rng.standard_normal((n, n))
