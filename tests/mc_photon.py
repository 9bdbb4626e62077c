"""Brute-force Monte Carlo photon transport in a uniform box, for pinning the
FP64 oracle's whole solver (test infrastructure; it shares nothing with the
oracle or the CUDA library).

The medium fills the box [0, lx] x [0, ly] x [0, lz] uniformly and moves with
a constant velocity beta (in units of c; beta = 0 is a static medium).  In
the medium's rest frame it absorbs with alpha0, scatters isotropically and
elastically with sigma0 (both grey), and emits isotropically with the energy
spectrum eta0(eps0) = A eps0^(-s) per unit volume, time, solid angle and
photon energy.  Faces are vacuum.

Packets stand for fixed numbers of photons and carry their laboratory-frame
energy.  Each is followed as a photon:
  * emission: a uniform point of the box, an isotropic rest-frame direction
    and a rest-frame photon energy drawn from eps0^(-s) on [e_lo, e_hi];
    direction and energy are Lorentz-transformed to the laboratory (the
    packet's energy scales with the photon's);
  * flight: straight in the laboratory with extinction chi_lab =
    (alpha0 + sigma0) Gamma (1 - beta . n) (the rest-frame extinction seen
    from the laboratory), an exponential optical depth per flight;
  * interaction: absorbed with probability alpha0/(alpha0 + sigma0), else
    transformed to the rest frame, given a new isotropic direction at the
    same rest-frame energy, and transformed back;
  * escape through any face.

The mean intensity in a tally cell is the path-length estimator
J = (rate per packet) * sum(E * l) / (4 pi V), per laboratory energy bin.
The emission rate in the laboratory equals the rest-frame one (emission
events per unit four-volume are invariant), so a packet of rest-frame energy
E0 stands for q0 V_box / N_packets events per unit time.
"""
from __future__ import annotations

import numpy as np


def _isotropic(rng, n):
    mu = rng.uniform(-1.0, 1.0, n)
    ph = rng.uniform(0.0, 2.0 * np.pi, n)
    st = np.sqrt(1.0 - mu * mu)
    return np.stack([st * np.cos(ph), st * np.sin(ph), mu], axis=1)


def _boost(n, beta):
    """Direction and photon-energy ratio eps_lab / eps_rest of a photon with
    rest-frame direction n seen from a frame in which the medium moves with
    velocity beta (textbook aberration and Doppler formulas)."""
    b2 = float(beta @ beta)
    if b2 == 0.0:
        return n.copy(), np.ones(len(n))
    gam = 1.0 / np.sqrt(1.0 - b2)
    bn = n @ beta
    dop = gam * (1.0 + bn)                      # eps_lab / eps_rest
    coef = (gam - 1.0) * bn / b2 + gam
    out = (n + coef[:, None] * beta[None, :]) / dop[:, None]
    out /= np.linalg.norm(out, axis=1)[:, None]
    return out, dop


def _unboost(n, beta):
    """The inverse of _boost: rest-frame direction of laboratory direction n
    and eps_rest / eps_lab."""
    return _boost(n, -beta)


def _cell_path(x0, d, t, lo, hi):
    """Length of the segments x0 + d [0, t] inside the box [lo, hi] (slab method)."""
    with np.errstate(divide="ignore", invalid="ignore"):
        inv = 1.0 / d
        t1 = (lo[None, :] - x0) * inv
        t2 = (hi[None, :] - x0) * inv
    tmin = np.where(np.isfinite(t1), np.minimum(t1, t2), -np.inf)
    tmax = np.where(np.isfinite(t1), np.maximum(t1, t2), np.inf)
    # a zero direction component: inside the slab or not at all
    flat = ~np.isfinite(t1)
    inside = (x0 >= lo[None, :]) & (x0 <= hi[None, :])
    tmin = np.where(flat & ~inside, np.inf, tmin)
    tmax = np.where(flat & ~inside, -np.inf, tmax)
    a = np.maximum(np.max(tmin, axis=1), 0.0)
    b = np.minimum(np.min(tmax, axis=1), t)
    return np.maximum(b - a, 0.0)


def _exit_distance(x, d, box):
    with np.errstate(divide="ignore", invalid="ignore"):
        tx = np.where(d > 0, (box[None, :] - x) / d, np.where(d < 0, -x / d, np.inf))
    return np.min(tx, axis=1)


def run(*, box, alpha0, sigma0, beta, A=1.0, s=0.0, e_lo=1.0, e_hi=1.0, cells, bins, n_packets, seed,
        batch=400_000, max_events=200):
    """Mean intensity and flux per laboratory energy bin in each tally cell.

    cells: list of (lo[3], hi[3]) boxes; bins: bin edges (laboratory photon
    energy; one bin [-inf, inf] for a grey problem with s = 0 and
    e_lo = e_hi).  Returns (M [4][cell][bin], standard error, same shape)
    with M[0] = J and M[1:4] = H_x, H_y, H_z (the first angular moments,
    divided by 4 pi like J), each the bin's integral over photon energy (the
    grey value for a single bin).  The error comes from the spread of
    independent batches.
    """
    rng = np.random.Generator(np.random.PCG64(seed))
    box = np.asarray(box, dtype=np.float64)
    beta = np.asarray(beta, dtype=np.float64)
    chi0 = alpha0 + sigma0
    gam = 1.0 / np.sqrt(1.0 - float(beta @ beta))
    vbox = float(np.prod(box))
    # rest-frame emitted power per unit volume: 4 pi A int eps^-s d eps
    if e_hi > e_lo:
        spec_int = (np.log(e_hi / e_lo) if s == 1.0 else (e_hi ** (1 - s) - e_lo ** (1 - s)) / (1 - s))
    else:
        spec_int = 1.0
    q0 = 4.0 * np.pi * A * spec_int
    E0 = q0 * vbox / n_packets                 # rest-frame energy of one packet (per unit time)
    nb = len(bins) - 1
    ncell = len(cells)
    sums = np.zeros((4, ncell, nb))
    sums2 = np.zeros((4, ncell, nb))
    nbatches = 0
    done = 0
    while done < n_packets:
        m = min(batch, n_packets - done)
        done += m
        nbatches += 1
        tally = np.zeros((4, ncell, nb))  # J, H_x, H_y, H_z
        x = rng.random((m, 3)) * box[None, :]
        n0 = _isotropic(rng, m)
        if e_hi > e_lo:
            u = rng.random(m)
            if s == 1.0:
                eps0 = e_lo * (e_hi / e_lo) ** u
            else:
                eps0 = (e_lo ** (1 - s) + u * (e_hi ** (1 - s) - e_lo ** (1 - s))) ** (1.0 / (1 - s))
        else:
            eps0 = np.full(m, e_lo)
        d, dop = _boost(n0, beta)
        eps = eps0 * dop
        E = E0 * dop
        alive = np.ones(m, dtype=bool)
        for _ in range(max_events):
            idx = np.nonzero(alive)[0]
            if idx.size == 0:
                break
            xa, da = x[idx], d[idx]
            chi_lab = chi0 * gam * (1.0 - da @ beta)
            tau = rng.exponential(1.0, idx.size)
            t_int = tau / chi_lab
            t_exit = _exit_distance(xa, da, box)
            t = np.minimum(t_int, t_exit)
            ea, Ea = eps[idx], E[idx]
            b = np.searchsorted(bins, ea) - 1
            okb = (b >= 0) & (b < nb)
            for ci, (lo, hi) in enumerate(cells):
                ell = _cell_path(xa, da, t, np.asarray(lo, float), np.asarray(hi, float))
                w = Ea * ell
                np.add.at(tally[0, ci], b[okb], w[okb])
                for q in range(3):
                    np.add.at(tally[1 + q, ci], b[okb], (w * da[:, q])[okb])
            escaped = t_exit <= t_int
            x[idx] = xa + t[:, None] * da
            # interactions
            inter = idx[~escaped]
            alive[idx[escaped]] = False
            if inter.size == 0:
                continue
            absorbed = rng.random(inter.size) < alpha0 / chi0
            alive[inter[absorbed]] = False
            sc = inter[~absorbed]
            if sc.size == 0:
                continue
            _, rest_over_lab = _unboost(d[sc], beta)   # eps_rest / eps_lab of the incoming photon
            eps_rest = eps[sc] * rest_over_lab
            E_rest = E[sc] * rest_over_lab
            nn, dop2 = _boost(_isotropic(rng, sc.size), beta)
            d[sc] = nn
            eps[sc] = eps_rest * dop2
            E[sc] = E_rest * dop2
        scale = n_packets / m  # this batch alone as an estimate of the whole run
        est = tally * scale
        sums += est
        sums2 += est * est
    vols = np.array([np.prod(np.asarray(hi, float) - np.asarray(lo, float)) for lo, hi in cells])
    mean = sums / nbatches
    var = np.maximum(sums2 / nbatches - mean * mean, 0.0) / max(1, nbatches - 1)
    J = mean / (4.0 * np.pi * vols[None, :, None])
    err = np.sqrt(var) / (4.0 * np.pi * vols[None, :, None])
    return J, err
