"""vlb_device_bytes (host-only arithmetic of the library, no GPU): the
footprint grows with the lattice, the particles and the storage width, and
inconsistent parameters are refused as vlb_create refuses them."""
import pytest


def _bytes(V, **over):
    radius = over.pop("radius", [8.0] * 16)
    p = V.vlb_params_default(**{"nx": 256, "ny": 256, "max_particles": len(radius), **over})
    return V.vlb_device_bytes(p, radius)


def test_footprint_orders():
    from paper_2410_23802_gb300 import vlb as V
    b32 = _bytes(V, precision=V.VLB_FP32)
    b16 = _bytes(V, precision=V.VLB_FP16_STORE)
    b64 = _bytes(V, precision=V.VLB_FP64)
    assert b16 < b32 < b64
    # per cell: 2 x 18 populations + 2 S planes + 7 macroscopic planes
    cells = 256 * 256
    assert 36 * 4 * cells + 9 * 4 * cells <= b32 < 36 * 4 * cells + 9 * 4 * cells + (2 << 20)
    assert _bytes(V, nx=512) > b32
    assert _bytes(V, radius=[8.0] * 32) > b32
    assert _bytes(V, radius=[12.0] * 16) > b32          # larger band tables
    assert _bytes(V, nx=250) == _bytes(V, nx=256)      # rows padded to 32 B
    assert _bytes(V, nx=248) < _bytes(V, nx=250)       # 248 needs no pad, 250 pads to 256


def test_footprint_refuses_bad_parameters():
    from paper_2410_23802_gb300 import vlb as V
    for over in ({"tau_f": 0.5}, {"nx": 1}, {"precision": 9}, {"rho_ratio": -1.0}):
        with pytest.raises(V.VlbError, match="EINVAL"):
            _bytes(V, **over)
    # no particles: the lattice alone
    p = V.vlb_params_default(nx=64, ny=64, max_particles=0)
    assert 0 < V.vlb_device_bytes(p, []) < _bytes(V, nx=64, ny=64)
