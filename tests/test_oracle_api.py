"""The oracle's C-ABI-shaped entry points (vlbref_*): the names and input
order of include/vlb.h, the same status codes, and exactly the results of
driving the oracle's Simulation directly."""
import inspect
import os
import re

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
CORE = ["create", "add_particles", "add_ellipses", "insert_particles", "set_fixed_temperature", "step", "get_fields", "get_particle_count",
        "get_particle_state", "get_audit", "get_step", "last_error", "destroy"]


def _header_params(name):
    text = re.sub(r"/\*.*?\*/", "", open(os.path.join(ROOT, "include", "vlb.h")).read(), flags=re.S)
    m = re.search(r"\bvlb_%s\s*\(([^)]*)\)" % name, text)
    return [re.findall(r"(\w+)\s*$", a.strip())[0] for a in m.group(1).split(",") if a.strip()]


def test_every_core_entry_point_has_an_oracle_twin():
    from oracle import vlbref as O
    for name in CORE:
        assert callable(getattr(O, "vlbref_" + name)), name
    # inputs in the header's order (the C out-parameters of scalars are returned instead)
    for name in ("add_particles", "add_ellipses", "insert_particles", "set_fixed_temperature", "step", "get_fields",
                 "get_particle_state"):
        py = list(inspect.signature(getattr(O, "vlbref_" + name)).parameters)
        assert py == _header_params(name), name


def test_oracle_api_equals_the_simulation():
    from oracle import vlbref as O
    from paper_2410_23802_gb300 import workloads as W
    case = W.cavity(side=96, n=6, seed=2, k_log_uniform=True)
    prm = O.Params(**{k: v for k, v in case.params.items() if k != "precision"})
    st, h = O.vlbref_create(prm)
    assert st == O.VLBREF_OK
    xy = np.column_stack([case.x, case.y]).reshape(-1)
    assert O.vlbref_add_particles(h, len(case.x), xy, case.radius, case.T0, case.k_ratio) == O.VLBREF_OK
    assert O.vlbref_step(h, 7) == O.VLBREF_OK
    n = O.vlbref_get_particle_count(h)[1]
    T = np.empty(96 * 96)
    assert O.vlbref_get_fields(h, O.VLBREF_FIELD_T, None, None, None, T, None) == O.VLBREF_OK
    xy_out, uv = np.empty(2 * n), np.empty(2 * n)
    assert O.vlbref_get_particle_state(h, n, xy_out, None, uv, None, None, None) == O.VLBREF_OK
    sim = O.Simulation(prm, case.x, case.y, case.radius, case.T0, k_ratio=case.k_ratio)
    sim.step(7)
    assert np.array_equal(T.reshape(96, 96), sim.fields()["T"])
    assert np.array_equal(xy_out[1::2], sim.particle_state()["y"])
    assert O.vlbref_get_step(h) == (O.VLBREF_OK, 7)
    assert O.vlbref_get_audit(h)[1:] == sim.audit()
    # the state rules of the C ABI
    assert O.vlbref_add_particles(h, 1, [30.0, 20.0], [3.0], [0.0]) == O.VLBREF_ESTATE
    O.vlbref_destroy(h)


def test_oracle_api_refuses_bad_disks():
    from oracle import vlbref as O
    st, h = O.vlbref_create(O.Params(nx=40, ny=40))
    assert O.vlbref_add_particles(h, 2, [20.0, 20.0, 25.0, 20.0], [4.0, 4.0], [0.0, 0.0]) == O.VLBREF_EINVAL
    assert "overlap" in O.vlbref_last_error(h)
    assert O.vlbref_add_particles(h, 1, [2.0, 20.0], [4.0], [0.0]) == O.VLBREF_EINVAL
    assert O.vlbref_create(O.Params(nx=40, ny=40, tau_f=0.5))[0] == O.VLBREF_EINVAL
