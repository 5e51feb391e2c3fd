"""The allocation-free solid-fraction entry point, through the C ABI.

vlb_get_solid_fraction_noalloc serves callers that cannot allocate device
memory during a run (a caching allocator or memory pool owns the device, or
cudaMalloc/cudaFree would synchronise it): it writes the same outputs as
vlb_get_solid_fraction from a static device scratch array of the library.
This test compares the two on two calls in a row, after a few steps so that
the particles have moved (both run the same dump kernel into buffers of the
same layout, so the outputs are identical bit for bit), checks that the call
leaves the device's free memory unchanged, and checks the size limit and the
state rule.  The file is collected last on purpose."""
import numpy as np
import pytest

from helpers import gpu_lattice
from paper_2410_23802_gb300 import workloads as W

pytestmark = pytest.mark.gpu


def _case(nx, ny):
    params = dict(nx=nx, ny=ny, tau_f=0.8, prandtl=0.7, rho_ratio=1.5, cv_ratio=2.0, k_ratio_default=3.0,
                  gravity=(0.0, -2e-5), beta=4.0, T_ref=1.0, T_fluid_init=1.0)
    xs = [20.0, 31.3, 55.75, 60.0, 80.2, 90.0]
    ys = [30.0, 32.5, 20.25, 40.0, 45.0, 20.0]
    rs = [5.0, 5.5, 6.0, 4.0, 7.5, 4.25]
    return W.Case("no-alloc", params, xs, ys, rs, [0.0, 0.2, 0.4, 0.6, 0.8, 1.0])


def _free_bytes():
    import torch
    torch.cuda.synchronize()
    return torch.cuda.mem_get_info()[0]


@pytest.mark.parametrize("precision", ["fp32", "fp64"])
def test_noalloc_matches_allocating_entry_point_twice(precision):
    from paper_2410_23802_gb300 import vlb as V
    nx, ny = 113, 67
    with gpu_lattice(_case(nx, ny), precision=precision) as lat:
        with pytest.raises(V.VlbError) as e:
            V.vlb_get_solid_fraction_noalloc(lat.h, nx, ny)  # no initial state yet
        assert e.value.status == V.VLB_ESTATE
        for call in range(2):
            lat.step(7)
            ref = V.vlb_get_solid_fraction(lat.h, nx, ny)
            V.vlb_synchronize(lat.h)
            free0 = _free_bytes()
            got = V.vlb_get_solid_fraction_noalloc(lat.h, nx, ny)
            free1 = _free_bytes()
            # an allocation would take at least one 2 MiB page of the device
            assert free0 - free1 < (2 << 20), (free0, free1)
            for a, b in zip(got, ref):
                np.testing.assert_array_equal(a, b)
            assert ref[0].max() >= 1


def test_noalloc_rejects_lattices_beyond_its_limit():
    from paper_2410_23802_gb300 import vlb as V
    nx, ny = 300, 300  # 90000 cells > VLB_NOALLOC_MAX_CELLS
    with gpu_lattice(_case(nx, ny), precision="fp32") as lat:
        lat.step(0)
        with pytest.raises(V.VlbError) as e:
            V.vlb_get_solid_fraction_noalloc(lat.h, nx, ny)
        assert e.value.status == V.VLB_EINVAL and "VLB_NOALLOC_MAX_CELLS" in str(e.value)
