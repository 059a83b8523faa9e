"""Parity rules shared by the GPU tests: the CUDA path against the FP64
oracle, one half-sweep layer at a time, and a record of what each check
excluded.

Tolerances:
  * every half-sweep layer is checked at every site of the updated colour:
    max |diff| <= 1e-5 per spin component at every site the two rules below
    do not exclude.  The record also counts the ill-conditioned sites, where
    4 kappa > 1e-5 with kappa = 2^-24 * sum_k |J_k| / |h| (the fp32 field's
    round-off relative to its length, which the update's direction
    inherits): at a nearly cancelling field no fp32 evaluation is bound to
    meet an absolute 1e-5, yet these sites are held to it too, and the
    record keeps their largest error;
  * Metropolis: sites whose accept decisions lie within 1e-5 of their
    threshold (|u3 - exp(-beta dE)| < 1e-5, margin reported by the oracle)
    are excluded (<= 0.2 % of them): fp32 and fp64 may decide differently;
  * heat-bath: sites whose field is within 1e-5 (relative) of the h_z = 0
    plane are excluded (<= 0.1 %): the orthonormal frame of the azimuth
    switches branch there and fp32/fp64 may pick different branches;
  * the colour not updated must stay bit-identical.
A sweep (colour 0, then colour 1, then more layers) is checked layer by
layer: layer k of the oracle starts from the GPU's own state after layer
k - 1, so each comparison measures one layer's error only; the GPU's
intermediate states come from half-sweeps issued one by one, which are
bit-identical to hsg_sweep (tested), or, for a single sweep of two layers,
from the final state itself (the colour-1 layer does not touch colour 0).

Every check appends what it measured to REPORT; with HSG_PARITY_REPORT set
to a path, the session writes REPORT there as JSON (tests/conftest.py).
"""
from __future__ import annotations

import numpy as np

import oracle

TOL = 1e-5
U32 = 2.0 ** -24
MET_NEAR_MAX = 0.002  # fraction of a colour's sites within 1e-5 of a Metropolis threshold
HB_BAND_MAX = 0.001  # fraction of a colour's sites in the heat-bath frame-branch band

REPORT: list[dict] = []


def colour_mask(L, c):
    g = np.indices((L, L, L))
    return (((g[0] + g[1] + g[2]) % 2) == c).reshape(-1)


def bond_sums(L, J):
    """sum of |J| over the six bonds of every site."""
    a = np.abs(np.asarray(J, dtype=np.float64).reshape(L, L, L, 3))  # [z, y, x, d]
    s = a.sum(axis=3)
    s += np.roll(a[..., 0], 1, axis=2) + np.roll(a[..., 1], 1, axis=1) + np.roll(a[..., 2], 1, axis=0)
    return s.reshape(-1)


def fields(L, Jr, state64, idx):
    return np.array([oracle.local_field(L, Jr, state64, int(i)) for i in idx]).reshape(-1, 3)


def check_half_sweep(L, Jr, before64, got, ref, colour, exclude=None, label="", max_excluded=None):
    """Compare one half-sweep site by site under the rules above; `exclude`
    marks sites the rules leave out (at most `max_excluded` of the colour).
    Returns the record appended to REPORT."""
    idx = np.nonzero(colour_mask(L, colour))[0]
    h = fields(L, Jr, before64, idx)
    hn = np.linalg.norm(h, axis=1)
    kappa = U32 * bond_sums(L, Jr)[idx] / np.maximum(hn, 1e-300)
    err = np.max(np.abs(np.asarray(got) - np.asarray(ref)).reshape(-1, 3)[idx], axis=1)
    skip = np.zeros(len(idx), bool) if exclude is None else np.asarray(exclude)[idx]
    well = (4 * kappa <= TOL) & ~skip
    ill = ~well & ~skip
    rec = dict(label=label, L=int(L), colour=int(colour), sites=int(len(idx)), excluded=int(skip.sum()),
               ill_conditioned=int(ill.sum()), max_err=float(err[~skip].max()) if (~skip).any() else 0.0,
               max_err_well=float(err[well].max()) if well.any() else 0.0,
               max_err_ill=float(err[ill].max()) if ill.any() else 0.0,
               max_err_over_kappa=float(np.max(err[~skip] / kappa[~skip])) if (~skip).any() else 0.0)
    REPORT.append(rec)
    if max_excluded is not None:
        assert skip.sum() <= max(2, max_excluded * len(idx)), rec
    assert np.all(err[~skip] <= TOL), rec
    return rec


def frame_band(L, Jr, before64, colour):
    """Sites whose field lies within 1e-5 (relative) of the h_z = 0 plane."""
    band = np.zeros(L ** 3, bool)
    idx = np.nonzero(colour_mask(L, colour))[0]
    h = fields(L, Jr, before64, idx)
    band[idx] = np.abs(h[:, 2]) < TOL * np.linalg.norm(h, axis=1)
    return band


def check_layer(L, Jr, before, after, upd, colour, params, label=""):
    """One half-sweep layer: the oracle applies update `upd` (oracle.OR, MET,
    HB or MET_OR) to colour `colour` of the GPU's state `before` (fp32
    values held in fp64); the GPU's `after` must agree under the rules
    above, and its other colour must equal `before` bit for bit."""
    before = np.asarray(before, dtype=np.float64)
    after = np.asarray(after, dtype=np.float64)
    ref = before.copy()
    mask = colour_mask(L, colour)
    exclude, cap = None, None
    if upd in (oracle.MET, oracle.MET_OR):
        margins = oracle.half_sweep(L, Jr, ref, upd, colour, params, want_margins=True)
        exclude, cap = mask & (margins < TOL), MET_NEAR_MAX
    else:
        oracle.half_sweep(L, Jr, ref, upd, colour, params)
        if upd == oracle.HB:
            exclude, cap = frame_band(L, Jr, before, colour), HB_BAND_MAX
    rec = check_half_sweep(L, Jr, before, after, ref, colour, exclude, label=label, max_excluded=cap)
    other = ~mask
    assert np.array_equal(after.reshape(-1, 3)[other], before.reshape(-1, 3)[other]), label
    return rec


def check_or_sweep(L, Jr, before, after, label=""):
    """One over-relaxation sweep (colour 0 then colour 1) from `before` to
    the GPU's `after`, layer by layer: colour 0 against the oracle's
    half-sweep of `before`; colour 1 against the oracle's half-sweep of the
    GPU's own new colour 0 beside the old colour 1 (the state the GPU's
    colour-1 layer started from)."""
    before = np.asarray(before, dtype=np.float64)
    after = np.asarray(after, dtype=np.float64)
    mid = np.where(np.repeat(colour_mask(L, 0), 3), after, before)
    p = oracle.Params()
    r0 = check_layer(L, Jr, before, mid, oracle.OR, 0, p, label=f"{label} OR c0")
    r1 = check_layer(L, Jr, mid, after, oracle.OR, 1, p, label=f"{label} OR c1")
    return r0, r1


def check_one_sweep(L, Jr, before, after, upd, params, label=""):
    """A sweep of one update kind (two layers: colour 0, then colour 1 at the
    same sweep counter), checked layer by layer as check_or_sweep does."""
    before = np.asarray(before, dtype=np.float64)
    after = np.asarray(after, dtype=np.float64)
    mid = np.where(np.repeat(colour_mask(L, 0), 3), after, before)
    r0 = check_layer(L, Jr, before, mid, upd, 0, params, label=f"{label} c0")
    r1 = check_layer(L, Jr, mid, after, upd, 1, params, label=f"{label} c1")
    return r0, r1


def record(**kw):
    """Append a free-form record (a sampled-site check, an energy error)."""
    REPORT.append(kw)
