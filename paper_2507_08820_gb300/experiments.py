"""Reduced-scale replications of the paper's equilibration-ratio results (Sec. III):
Table III and the wavevector-resolved spectra of Figs. 1 and 2.

Table III: for each relaxation time the fluid starts at rest (or in the thermal state),
thermalises, and the per-site variances of rho, rho u, the diagonal and the off-diagonal
second Hermite moment (Pi) are averaged over snapshots (FP64 per-mode sums on the GPU,
`rflbm_mode_sums`). The equilibration ratio (Sec. III) is the measured variance over the
fluctuation-dissipation value rho0 kT b_k / cs2 summed over the components, the
conserved ones times (1 - 1/N).

Figs. 1 and 2: the same ratios per spherical shell of wavevectors, from the static
structure factors S(|k|) of the ten fields (cuFFT of each snapshot, shell sums on the
GPU, `rflbm_structure_factor`) averaged over snapshots and divided by their flat
fluctuation-dissipation values rho0 kT / cs2, rho0 kT, 2 rho0 kT cs2 and rho0 kT cs2. Fig. 1
is the spectrum of the four ratios for both models at tau = 0.51 and 50; Fig. 2 the
minimum and maximum over shells of ER(sum rho u) against tau.

A run whose state goes non-finite is reported as unstable, as the paper does for the
BGK model below tau = 0.505.

    python -m paper_2507_08820_gb300.experiments [table3|fig1|fig2] [--edge 128] [--steps 20000]
        [--burn 5000] [--start rest|thermal] [--json]
"""
from __future__ import annotations

import argparse
import json
import sys

import numpy as np

TABLE3_TAUS = (0.5001, 0.5005, 0.501, 0.505, 0.51, 0.55, 0.7, 1.0, 1.5, 2.0, 5.0, 10.0, 50.0, 100.0)
# Table II norms b_k of the modes rho, j (3), Pi_aa (3), Pi_ab (3)
_B = np.array([1.0, 1 / 3, 1 / 3, 1 / 3, 2 / 9, 2 / 9, 2 / 9, 1 / 9, 1 / 9, 1 / 9])


def _box(R, edge, tau, kT, model, seed, storage, start, phi_rho="local"):
    box = R.Box(edge, edge, edge, tau=tau, kT=kT, seed=seed, storage=storage,
                model=R.RFLBM_MODEL_BGK if model == "bgk" else R.RFLBM_MODEL_REG,
                phi_rho=R.RFLBM_PHI_RHO0 if phi_rho == "rho0" else R.RFLBM_PHI_LOCAL_RHO)
    (R.rflbm_init_thermal if start == "thermal" else R.rflbm_init_rest)(box.h)
    return box


def equilibration_ratios(tau, kT=1.0 / 3000.0, model="reg", edge=128, steps=20000, burn=5000,
                         every=100, seed=1, storage=0, start="rest", phi_rho="local"):
    """ER(rho), ER(sum rho u), ER(sum Pi_aa), ER(sum Pi_a<b) of one run, or None when the
    run became non-finite. phi_rho: the density in Eq. 10, "local" or "rho0"."""
    from paper_2507_08820_gb300 import rflbm as R
    n = edge ** 3
    box = _box(R, edge, tau, kT, model, seed, storage, start, phi_rho)
    try:
        R.rflbm_step(box.h, burn)
        var = np.zeros(10)
        snaps = 0
        for _ in range(burn, steps, every):
            R.rflbm_step(box.h, every)
            st, status = R.rflbm_stats(box.h)
            if status == R.RFLBM_EUNSTABLE:
                return None
            s1, s2 = R.rflbm_mode_sums(box.h)
            var += s2[:10] / n - (s1[:10] / n) ** 2
            snaps += 1
        var /= max(snaps, 1)
    finally:
        box.close()
    theory = 3.0 * kT * _B
    theory[:4] *= 1.0 - 1.0 / n
    return (var[0] / theory[0], var[1:4].sum() / theory[1:4].sum(),
            var[4:7].sum() / theory[4:7].sum(), var[7:10].sum() / theory[7:10].sum())


def table3(taus=TABLE3_TAUS, models=("reg", "bgk"), **kw):
    """{model: {tau: (ER...) or None}}."""
    return {m: {tau: equilibration_ratios(tau, model=m, **kw) for tau in taus} for m in models}


# flat structure factors of the ten fields per unit rho0 kT: rho, rho u (3), Pi_aa (3),
# Pi_a<b (3), i.e. b_k / cs2 of their modes
_S_THEORY = np.array([3.0, 1.0, 1.0, 1.0, 2 / 3, 2 / 3, 2 / 3, 1 / 3, 1 / 3, 1 / 3])
_GROUPS = ((0,), (1, 2, 3), (4, 5, 6), (7, 8, 9))


def er_spectra(tau, kT=1.0 / 3000.0, model="reg", edge=128, steps=20000, burn=0, every=100,
               seed=1, storage=0, start="thermal", phi_rho="local"):
    """Per-shell equilibration ratios (Fig. 1): an array (4, nshell) of ER(rho),
    ER(sum rho u), ER(sum Pi_aa), ER(sum Pi_a<b) for shells n = round(|k| L / 2 pi), and the
    number of wavevectors per shell; None when the run became non-finite."""
    from paper_2507_08820_gb300 import rflbm as R
    box = _box(R, edge, tau, kT, model, seed, storage, start, phi_rho)
    try:
        ns = R.rflbm_shell_count(box.h)
        acc = np.zeros((10, ns))
        count = None
        snaps = 0
        R.rflbm_step(box.h, burn)
        for _ in range(burn, steps, every):
            R.rflbm_step(box.h, every)
            st, status = R.rflbm_stats(box.h)
            if status == R.RFLBM_EUNSTABLE:
                return None
            for f in range(10):
                s, count = R.rflbm_structure_factor(box.h, f, ns)
                acc[f] += s
            snaps += 1
    finally:
        box.close()
    with np.errstate(invalid="ignore", divide="ignore"):
        per_field = acc / snaps / np.where(count > 0, count, np.nan)[None, :]
    er = np.array([per_field[list(g)].sum(axis=0) / (kT * _S_THEORY[list(g)].sum()) for g in _GROUPS])
    return er, count


def fig1(edge=128, **kw):
    """{(model, tau): ER spectra} for both models at tau = 0.51 and 50 (Fig. 1)."""
    return {(m, t): er_spectra(t, model=m, edge=edge, **kw) for m in ("bgk", "reg") for t in (0.51, 50.0)}


def fig2(taus=TABLE3_TAUS, edge=128, shells=None, **kw):
    """{model: {tau: (min, max) of ER(sum rho u) over the shells, or None}} (Fig. 2). The
    paper scores shells 4 <= |k| <= 64 of its 256^3 box; `shells` defaults to the same
    wavelengths at this edge."""
    lo, hi = shells if shells else (max(1, edge // 64), edge // 4)
    out = {}
    for m in ("reg", "bgk"):
        out[m] = {}
        for t in taus:
            r = er_spectra(t, model=m, edge=edge, **kw)
            out[m][t] = None if r is None else (float(np.min(r[0][1, lo:hi + 1])), float(np.max(r[0][1, lo:hi + 1])))
    return out


def main(argv=None):
    ap = argparse.ArgumentParser(description=__doc__.split("\n\n")[0])
    ap.add_argument("what", nargs="?", choices=["table3", "fig1", "fig2"], default="table3")
    ap.add_argument("--edge", type=int, default=128)
    ap.add_argument("--steps", type=int, default=20000)
    ap.add_argument("--burn", type=int, default=None, help="default: 5000 from rest, 0 thermal")
    ap.add_argument("--every", type=int, default=100)
    ap.add_argument("--kT", type=float, default=1.0 / 3000.0)
    ap.add_argument("--start", choices=["rest", "thermal"], default=None,
                    help="default: rest for table3, thermal for the spectra")
    ap.add_argument("--phi-rho", choices=["local", "rho0"], default="local",
                    help="density in the noise amplitude of Eq. 10")
    ap.add_argument("--json", action="store_true")
    a = ap.parse_args(argv)
    from paper_2507_08820_gb300 import build
    build.build()
    start = a.start or ("rest" if a.what == "table3" else "thermal")
    burn = a.burn if a.burn is not None else (5000 if start == "rest" else 0)
    kw = dict(edge=a.edge, steps=a.steps, burn=burn, every=a.every, kT=a.kT, start=start, phi_rho=a.phi_rho)
    if a.what != "table3":
        return _main_spectra(a, kw)
    res = table3(**kw)
    if a.json:
        print(json.dumps({m: {str(t): v for t, v in r.items()} for m, r in res.items()}))
        return 0
    print(f"# equilibration ratios, {a.edge}^3, kT = {a.kT:.6g}, {a.steps} steps "
          f"(start {start}, burn-in {burn}, snapshot every {a.every}, rho of Eq. 10: {a.phi_rho}); "
          "Reg-FLBM (BGK-FLBM)")
    print("tau      ER(rho)          ER(sum rho u)    ER(sum Pi_aa)    ER(sum Pi_a<b)")
    for tau in TABLE3_TAUS:
        reg, bgk = res["reg"][tau], res["bgk"][tau]
        cols = []
        for i in range(4):
            r = f"{reg[i]:.4f}" if reg else "  ... "
            b = f"({bgk[i]:.4f})" if bgk else "(...)"
            cols.append(f"{r} {b:9s}")
        print(f"{tau:<8g} " + "  ".join(cols))
    return 0


def _main_spectra(a, kw):
    names = ("ER(rho)", "ER(sum rho u)", "ER(sum Pi_aa)", "ER(sum Pi_a<b)")
    if a.what == "fig1":
        res = fig1(**kw)
        if a.json:
            print(json.dumps({f"{m} {t:g}": None if r is None else {"er": r[0].tolist(), "count": r[1].tolist()}
                              for (m, t), r in res.items()}))
            return 0
        lo, hi = max(1, a.edge // 64), a.edge // 4
        bands = [(lo, 2 * lo), (2 * lo, 4 * lo), (4 * lo, 8 * lo), (8 * lo, hi + 1)]
        print(f"# ER spectra, {a.edge}^3, kT = {a.kT:.6g}, {a.steps} steps, start {kw['start']}: "
              "mean of each shell band [n0, n1)")
        for (m, t), r in res.items():
            if r is None:
                print(f"{m} tau {t:g}: unstable")
                continue
            er, count = r
            for f, name in enumerate(names):
                cells = [np.nansum(er[f, b0:b1] * count[b0:b1]) / count[b0:b1].sum() for b0, b1 in bands]
                print(f"{m} tau {t:<5g} {name:15s} " + "  ".join(f"[{b0},{b1}) {c:.4f}" for (b0, b1), c in zip(bands, cells)))
        return 0
    res = fig2(**kw)
    if a.json:
        print(json.dumps({m: {str(t): v for t, v in r.items()} for m, r in res.items()}))
        return 0
    print(f"# min / max of ER(sum rho u) over shells, {a.edge}^3, kT = {a.kT:.6g}, {a.steps} steps, "
          f"start {kw['start']}; Reg-FLBM (BGK-FLBM)")
    for t in TABLE3_TAUS:
        cols = []
        for m in ("reg", "bgk"):
            v = res[m][t]
            cols.append("unstable" if v is None else f"{v[0]:.4f} / {v[1]:.4f}")
        print(f"{t:<8g} {cols[0]:>20s}   ({cols[1]})")
    return 0


if __name__ == "__main__":
    sys.exit(main())
