"""The allocation-free P(k) entry point against the context version.

pm_power_spectrum_noalloc serves callers that cannot call cudaMalloc where
they want the diagnostic (an allocator that forbids further allocation, or
device memory handed entirely to the application's own sub-allocator).  It
runs on a fixed scratch array inside the library, so after its first call on
a device it must not change the device's free memory, and two calls in a row
must both reproduce pm_power_spectrum of a context holding the same particles.
The mesh sizes cover the generic mixed-radix FFT path (8, 24, 48, whose
twiddles the entry point computes on the device) and the compiled passes
(32, 64).  This file is collected last on purpose.
"""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu

OM, BOX = 0.31, 320.0


@pytest.mark.parametrize("n,npart_side", [(8, 6), (24, 13), (32, 32), (48, 17), (64, 20)])
def test_noalloc_power_spectrum_matches_context_version(n, npart_side):
    import torch
    from paper_2607_17929_gb300 import build
    build.build()
    from paper_2607_17929_gb300 import ics, pm

    nbins = n // 2 - 2
    pos, mom = ics.zeldovich_ics(npart_side, BOX * npart_side / n, OM, 0.67, 1 / 101, 1 / 101, 11 + n)
    ctx = pm.PM(n, npart_side ** 3, BOX, OM, 100.0, 0.0, 100, pm.PM_FP64)
    ctx.set_particles(pos, mom)
    k0, pk0, nm0 = ctx.power_spectrum(nbins)
    ctx.close()

    d_pos = torch.from_numpy(pos).cuda()
    stream = torch.cuda.current_stream()
    torch.cuda.synchronize()
    results = [pm.pm_power_spectrum_noalloc(d_pos, n, OM, nbins, stream)]  # first call: per-device set-up
    torch.cuda.synchronize()
    free_before, _ = torch.cuda.mem_get_info()
    results.append(pm.pm_power_spectrum_noalloc(d_pos, n, OM, nbins, stream))
    torch.cuda.synchronize()
    free_after, _ = torch.cuda.mem_get_info()
    assert free_after == free_before
    for k, pk, nm in results:
        assert np.array_equal(nm, nm0)
        rel = np.linalg.norm(pk[1:] - pk0[1:]) / np.linalg.norm(pk0[1:])
        assert rel < 1e-11, rel
        assert np.max(np.abs(k[1:] - k0[1:]) / k0[1:]) < 1e-13


def test_noalloc_rejects_sizes_above_its_scratch():
    import torch
    from paper_2607_17929_gb300 import pm

    d_pos = torch.rand((100, 3), dtype=torch.float64, device="cuda")
    with pytest.raises(pm.PMError) as e:
        pm.pm_power_spectrum_noalloc(d_pos, 128, OM, 8)
    assert e.value.status == pm.PM_ERR_UNSUPPORTED_SIZE
    with pytest.raises(pm.PMError) as e:
        pm.pm_power_spectrum_noalloc(d_pos, 32, OM, 4096)
    assert e.value.status == pm.PM_ERR_UNSUPPORTED_SIZE
    # host memory of the right layout reaches the library, which rejects it
    with pytest.raises(pm.PMError) as e:
        pm.pm_power_spectrum_noalloc(d_pos.cpu().numpy(), 32, OM, 8)
    assert e.value.status == pm.PM_ERR_INVALID_ARG
