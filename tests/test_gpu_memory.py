"""Device memory comes back: building B (whitening scratch, slices) and running a split-precision SCF on
handle after handle must not leave allocations behind (many-molecule runs would exhaust HBM)."""
import pytest

from paper_1707_03771_gb300 import clusters

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def lib():
    from paper_1707_03771_gb300 import binding, build
    build.build()
    return binding


def test_handles_release_device_memory(lib):
    import torch
    system = clusters.workload("water8")
    with lib.Handle(system) as h:          # first use: library state, autotuner choices, tile timings
        h.build_B()
        h.scf(precision=lib.DF_PREC_SPLIT, slices=3, incremental=1)
    torch.cuda.synchronize()
    free0 = torch.cuda.mem_get_info()[0]
    for _ in range(3):
        with lib.Handle(system) as h:
            h.build_B()
            r = h.scf(precision=lib.DF_PREC_SPLIT, slices=3, incremental=1)
            assert r["converged"]
    torch.cuda.synchronize()
    free1 = torch.cuda.mem_get_info()[0]
    print(f"free before {free0 / 1e9:.3f} GB, after {free1 / 1e9:.3f} GB")
    assert free0 - free1 < 64 << 20
