"""Reduced-scale replication of the paper's equilibration-ratio table (Table III).

For each relaxation time the fluid starts at rest, thermalises, and the per-site
variances of rho, rho u, the diagonal and the off-diagonal second Hermite moment (Pi) are
averaged over snapshots (FP64 per-mode sums on the GPU, `rflbm_mode_sums`). The
equilibration ratio (Sec. III) is the measured variance over the fluctuation-dissipation
value rho0 kT b_k / cs2 summed over the components, the conserved ones times (1 - 1/N).
A run whose state goes non-finite is reported as unstable, as the paper does for the
BGK model below tau = 0.505.

    python -m paper_2507_08820_gb300.experiments [--edge 128] [--steps 20000] [--burn 5000]
"""
from __future__ import annotations

import argparse
import json
import sys

import numpy as np

TABLE3_TAUS = (0.5001, 0.5005, 0.501, 0.505, 0.51, 0.55, 0.7, 1.0, 1.5, 2.0, 5.0, 10.0, 50.0, 100.0)
# Table II norms b_k of the modes rho, j (3), Pi_aa (3), Pi_ab (3)
_B = np.array([1.0, 1 / 3, 1 / 3, 1 / 3, 2 / 9, 2 / 9, 2 / 9, 1 / 9, 1 / 9, 1 / 9])


def equilibration_ratios(tau, kT=1.0 / 3000.0, model="reg", edge=128, steps=20000, burn=5000,
                         every=100, seed=1, storage=0):
    """ER(rho), ER(sum rho u), ER(sum Pi_aa), ER(sum Pi_a<b) of one run, or None when the
    run became non-finite."""
    from paper_2507_08820_gb300 import rflbm as R
    n = edge ** 3
    box = R.Box(edge, edge, edge, tau=tau, kT=kT, seed=seed, storage=storage,
                model=R.RFLBM_MODEL_BGK if model == "bgk" else R.RFLBM_MODEL_REG)
    try:
        R.rflbm_init_rest(box.h)
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


def main(argv=None):
    ap = argparse.ArgumentParser(description=__doc__.split("\n\n")[0])
    ap.add_argument("--edge", type=int, default=128)
    ap.add_argument("--steps", type=int, default=20000)
    ap.add_argument("--burn", type=int, default=5000)
    ap.add_argument("--every", type=int, default=100)
    ap.add_argument("--kT", type=float, default=1.0 / 3000.0)
    ap.add_argument("--json", action="store_true")
    a = ap.parse_args(argv)
    from paper_2507_08820_gb300 import build
    build.build()
    res = table3(edge=a.edge, steps=a.steps, burn=a.burn, every=a.every, kT=a.kT)
    if a.json:
        print(json.dumps({m: {str(t): v for t, v in r.items()} for m, r in res.items()}))
        return 0
    print(f"# equilibration ratios, {a.edge}^3, kT = {a.kT:.6g}, {a.steps} steps "
          f"(burn-in {a.burn}, snapshot every {a.every}); Reg-FLBM (BGK-FLBM)")
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


if __name__ == "__main__":
    sys.exit(main())
