"""Test-only glue: the same seeded case fed to the CUDA path and the oracle."""
import numpy as np

PREC = {"fp64": 0, "fp32": 1, "fp16": 2, "bf16": 3}  # VLB_FP64, VLB_FP32, VLB_FP16_STORE, VLB_BF16_STORE


def gpu_lattice(case, precision=None, max_particles=None, **over):
    from paper_2410_23802_gb300 import vlb as V
    prm = dict(case.params)
    prm.update(over)
    prec = PREC[precision or prm.pop("precision", "fp32")]
    prm.pop("precision", None)
    n = len(case.x)
    p = V.vlb_params_default(precision=prec, max_particles=max_particles or max(n, 1), **prm)
    lat = V.Lattice(p)
    if n and getattr(case, "semi_minor", None) is not None:
        lat.add_ellipses(np.column_stack([case.x, case.y]), case.radius, case.semi_minor, case.theta0, case.T0,
                         k_ratio=case.k_ratio)
    elif n:
        xy = np.column_stack([case.x, case.y])
        lat.add_particles(xy, case.radius, case.T0, k_ratio=case.k_ratio)
        if getattr(case, "fixed_T", None) is not None:
            V.vlb_set_fixed_temperature(lat.h, case.fixed_T)
    return lat


def oracle_sim(case, **over):
    from oracle import vlbref as O
    prm = {k: v for k, v in case.params.items() if k != "precision"}
    prm.update(over)
    for key in ("periodic", "outflow"):
        if key in prm:
            prm[key] = tuple(bool(v) for v in prm[key])
    return O.Simulation(O.Params(**prm), case.x, case.y, case.radius, case.T0, k_ratio=case.k_ratio,
                        fixed_T=getattr(case, "fixed_T", None), semi_minor=getattr(case, "semi_minor", None),
                        theta=getattr(case, "theta0", None))


def rel_l2(a, b):
    a = np.asarray(a, dtype=np.float64)
    b = np.asarray(b, dtype=np.float64)
    return float(np.sqrt(((a - b) ** 2).sum() / max((b ** 2).sum(), 1e-300)))
