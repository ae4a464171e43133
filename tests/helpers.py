"""Shared set-up for the parity tests: oracle problems and seeded inputs."""
from __future__ import annotations

import json
import os

import numpy as np

import oracle as O
import synth


def oracle_problem(scan, rcond_min=1e-3):
    """Oracle view of a scan after the pixel selection (samples of dropped pixels flagged)."""
    prob = O.Problem.from_scan(scan)
    blocks, hits = O.bd_blocks(prob)
    good = O.select_pixels(blocks, hits, rcond_min)
    prob = prob.with_pix(O.flag_samples(prob.pix, good))
    blocks, _ = O.bd_blocks(prob)
    mbd = O.bd_inverse(blocks, good)
    return prob, mbd, good


def truncated_problem(scan, length, rcond_min=1e-3, good=None):
    """Oracle problem of the first `length` samples of every detector timeline.

    Pixel selection comes from the full scan (``good``), as in the library.
    """
    keep = (np.arange(scan.n_samples) % scan.n_t) < length
    pix = scan.pix.astype(np.int64).copy()
    if good is not None:
        ok = pix >= 0
        bad = np.zeros_like(ok)
        bad[ok] = ~good[pix[ok]]
        pix[bad] = -1
    offs = []
    bands = []
    for b in range(scan.n_blocks):
        o0, o1 = int(scan.block_off[b]), int(scan.block_off[b + 1])
        d0 = (o0 // scan.n_t) * scan.n_t
        hi = min(o1, d0 + length)
        if hi > o0:
            offs.append((o0, hi))
            bands.append(scan.block_band[b])
    idx = np.concatenate([np.arange(a, b) for a, b in offs])
    new_off = np.concatenate([[0], np.cumsum([b - a for a, b in offs])])
    prob = O.Problem(pix[idx], scan.psi[idx], new_off, scan.band, np.array(bands), scan.n_pix)
    blocks, hits = O.bd_blocks(prob)
    g = good if good is not None else O.select_pixels(blocks, hits, rcond_min)
    # a pixel kept on the full scan but numerically singular in this prefix
    # gets a zero M_BD block (as in the library), so PCG leaves it at zero
    ev = np.linalg.eigvalsh(blocks)
    with np.errstate(divide="ignore", invalid="ignore"):
        rc = np.where(ev[:, 2] > 0, ev[:, 0] / ev[:, 2], 0.0)
    mbd = O.bd_inverse(blocks, g & (hits > 0) & (rc > 1e-12))
    return prob, mbd, idx


def rel(a, b):
    a = np.asarray(a, dtype=np.float64).reshape(-1)
    b = np.asarray(b, dtype=np.float64).reshape(-1)
    nb = np.linalg.norm(b)
    return np.linalg.norm(a - b) / (nb if nb > 0 else 1.0)


STOKES = ("I", "Q", "U")


def stokes_errors(a, ref):
    """Errors of a map (or of rows of A x) against a reference, per Stokes column c = I, Q, U.

    norm[c]: ||a_c - ref_c|| / ||ref_c||, the relative 2-norm of one column;
    elem[c]: max_i |a_ic - ref_ic| / max(|ref_ic|, s_c), every element against its own value,
             floored at the column's scale s_c = rms(ref_c) so that entries near zero are judged
             against the size of the column rather than against themselves.
    A column that is zero in the reference (Q, U of an intensity-only map) is judged against the
    scale of the whole array.  Also returns the whole-array relative 2-norm.
    """
    a = np.asarray(a, dtype=np.float64).reshape(-1, 3)
    r = np.asarray(ref, dtype=np.float64).reshape(-1, 3)
    assert a.shape == r.shape, (a.shape, r.shape)
    total = np.sqrt(np.mean(r * r)) if r.size else 0.0
    out = {"total": rel(a, r), "norm": {}, "elem": {}, "worst": {}}
    for c, name in enumerate(STOKES):
        rc, ac = r[:, c], a[:, c]
        s = np.sqrt(np.mean(rc * rc)) if rc.size else 0.0
        if s == 0.0:
            s = total if total > 0 else 1.0
            out["norm"][name] = float(np.linalg.norm(ac - rc) / (s * np.sqrt(max(rc.size, 1))))
        else:
            out["norm"][name] = float(np.linalg.norm(ac - rc) / np.linalg.norm(rc))
        e = np.abs(ac - rc) / np.maximum(np.abs(rc), s)
        i = int(np.argmax(e)) if e.size else 0
        out["elem"][name] = float(e[i]) if e.size else 0.0
        out["worst"][name] = i
    return out


def assert_close(a, ref, tol, what="", elem_tol=None):
    """Parity of the CUDA path with the oracle (or of two CUDA results) at tolerance `tol`:
    the whole-array relative 2-norm, every Stokes column's relative 2-norm and every element
    (see stokes_errors) must each stay within tol (elements within elem_tol when given).  With
    MM_PARITY_LOG set, the errors are appended to that file as one JSON line per check."""
    etol = tol if elem_tol is None else elem_tol
    e = stokes_errors(a, ref)
    log = os.environ.get("MM_PARITY_LOG")
    if log:
        test = os.environ.get("PYTEST_CURRENT_TEST", "").split(" ")[0]
        with open(log, "a") as f:
            f.write(json.dumps({"test": test, "what": what, "tol": tol, "elem_tol": etol, **e}) + "\n")
    bad = [f"norm[{c}]={e['norm'][c]:.3e}" for c in STOKES if not e["norm"][c] <= tol]
    bad += [f"elem[{c}]={e['elem'][c]:.3e}" for c in STOKES if not e["elem"][c] <= etol]
    assert e["total"] <= tol and not bad, (
        f"{what}: total {e['total']:.3e}, " + ", ".join(bad or ["-"]) + f" above {tol:g} / {etol:g} (worst elements "
        + ", ".join(f"{c}@{e['worst'][c]}" for c in STOKES) + ")")


def scan_and_tod(name_or_cfg, seed=0, sky=True, noise=True, **over):
    if isinstance(name_or_cfg, str):
        scan = synth.scan_from_config(name_or_cfg, seed=seed, **over)
    else:
        cfg = dict(name_or_cfg)
        cfg.update(over)
        scan = synth.make_scan(seed=seed, **cfg)
    s = synth.make_sky(scan.n_pix, seed) if sky else None
    n = synth.make_noise(scan, seed) if noise else None
    d = synth.make_tod(scan, s, n)
    return scan, d, s
