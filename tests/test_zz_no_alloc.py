"""rt_energy_static: the energy sum for callers that may not allocate device memory (a host
code whose pool owns the GPU, a monitoring hook).  Its partial sums live in a fixed array of
the library's device memory; it must agree with rt_energy, call after call."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

from paper_2302_12727_gb300 import (RT_ENERGY_STATIC_MAX_GROUPS, RT_FP32_MIXED, RT_FP64, RTError,  # noqa: E402
                                    Transport, rt_energy_static, workloads as W)

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("precision", ["fp64", "fp32"])
def test_energy_static_matches_rt_energy_on_consecutive_calls(precision):
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    rng = np.random.default_rng(77)
    x = W.jittered_lattice(14, 0.2, rng)
    n = x.shape[1]
    G = 3
    t = Transport(x, None, None, n_groups=G, precision=precision)
    V = t.fields()["V"]
    prec = RT_FP64 if precision == "fp64" else RT_FP32_MIXED
    stream = torch.cuda.current_stream().cuda_stream
    out = torch.full((G,), float("nan"), dtype=torch.float64, device="cuda")
    for call in range(2):
        # a different state each call: nothing of the previous call may leak into this one
        U0 = np.zeros((G, 4, n))
        U0[:, 0] = rng.uniform(0.5, 2.0 + call, size=(G, n))
        U0[:, 1:] = rng.normal(size=(G, 3, n))
        U = t.state(U0)
        want = np.array(t.energy(U))
        rt_energy_static(U, V, n, G, prec, out, stream)
        torch.cuda.synchronize()
        got = out.cpu().numpy()
        # both sum in double; only the order of the summation differs
        np.testing.assert_allclose(got, want, rtol=1e-13)
    # after those calls (the first loaded the array), a further call leaves the device's free
    # memory exactly where it was: it allocated nothing, directly or through the driver
    torch.cuda.synchronize()
    free0, _ = torch.cuda.mem_get_info()
    rt_energy_static(U, V, n, G, prec, out, stream)
    torch.cuda.synchronize()
    free1, _ = torch.cuda.mem_get_info()
    assert free1 == free0
    np.testing.assert_allclose(out.cpu().numpy(), want, rtol=1e-13)
    t.close()


def test_energy_static_rejects_too_many_groups():
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    G = RT_ENERGY_STATIC_MAX_GROUPS + 1
    U = torch.zeros(4 * G * 8, dtype=torch.float64, device="cuda")
    V = torch.ones(8, dtype=torch.float64, device="cuda")
    out = torch.zeros(G, dtype=torch.float64, device="cuda")
    with pytest.raises(RTError, match="RT_ERR_INVALID"):
        rt_energy_static(U, V, 8, G, RT_FP64, out)
