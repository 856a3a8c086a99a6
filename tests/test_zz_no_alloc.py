"""df_coulomb_noalloc: the Coulomb build for callers that cannot allocate device memory.

Some callers cannot call cudaMalloc (an application that owns all device memory through its own
allocator, or a loop that cannot afford an allocation's synchronisation). This entry point takes its
scratch from a fixed array inside the library; here its J is checked against the J of the regular
entry point df_jk, within the tolerance of the other J/K kernel tests, on two calls in a row with
different densities (the shared scratch keeps the previous call's contents), and the device's free
memory is read before and after each call: the handle resolved the scratch array (and loaded the kernels)
when it was created, so neither the first call nor the second may take any device memory.

Collected last so that a run stopping at its first failure has already run every other test.
"""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu

TOL = 1e-12   # relative to max |J|, as in the J/K kernel parity test


@pytest.fixture(scope="module")
def env():
    torch = pytest.importorskip("torch")
    from paper_1707_03771_gb300 import binding, build, clusters
    build.build()
    return torch, binding, clusters


@pytest.mark.parametrize("name", ["water2", "water8"])
def test_noalloc_coulomb_matches_df_jk_twice(env, name):
    torch, binding, clusters = env
    system = clusters.workload(name)
    dev = torch.device("cuda", 0)
    rng = np.random.default_rng(11)
    with binding.Handle(system) as h:
        h.build_B()
        for call in range(2):
            C = rng.normal(size=(h.n, h.nocc)) * (0.2 + 0.1 * call)
            D = 2 * C @ C.T
            J_ref, _ = h.jk(D, C)
            dD = torch.from_numpy(D).to(dev)
            dJ = torch.full((h.n, h.n), float("nan"), dtype=torch.float64, device=dev)
            torch.cuda.synchronize()          # D is on the device before the library's stream reads it
            free_before = torch.cuda.mem_get_info(dev)[0]
            h.coulomb_noalloc(dD.data_ptr(), dJ.data_ptr())
            torch.cuda.synchronize()          # the call only enqueues work
            free_after = torch.cuda.mem_get_info(dev)[0]
            assert free_after == free_before, (name, call, free_before - free_after)
            J = dJ.cpu().numpy()
            assert np.all(np.isfinite(J)), (name, call)
            assert np.abs(J - J_ref).max() <= TOL * np.abs(J_ref).max(), (name, call)


def test_noalloc_rejects_systems_beyond_the_static_scratch(env):
    torch, binding, clusters = env
    system = clusters.water_cluster(52, 52)       # n = 2600: needs more than 48 MiB of scratch
    dev = torch.device("cuda", 0)
    dummy = torch.zeros(4, dtype=torch.float64, device=dev)
    with binding.Handle(system) as h:
        with pytest.raises(binding.DFError) as e:
            h.coulomb_noalloc(dummy.data_ptr(), dummy.data_ptr())
        assert e.value.code == binding.DF_E_ARG
        assert "static maximum" in str(e.value)
