"""bdm_set_agents on the device: the positions go into both position buffers
(the iteration's parity picks the one read), and every input that is not a
finite position within +-1e9 um or a finite diameter in (0, 1e6) um is refused
with BDM_EINVAL and leaves no agents set, from host and from device memory."""
import numpy as np
import pytest

from paper_2301_06984_gb300 import bdm

pytestmark = pytest.mark.gpu


@pytest.fixture(autouse=True, scope="module")
def _cuda():
    import torch
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    yield


def _agents(n=5000, seed=5):
    rng = np.random.default_rng(seed)
    p = rng.uniform(-300.0, 300.0, (3, n))
    d = rng.uniform(8.0, 12.0, n)
    return p[0].copy(), p[1].copy(), p[2].copy(), d


def _as(mem, a):
    if mem == "host":
        return a
    import torch
    return torch.as_tensor(a, device="cuda")


@pytest.mark.parametrize("mem", ["host", "device"])
@pytest.mark.parametrize("step", [0, 1])
def test_positions_in_both_buffers(mem, step):
    x, y, z, d = _agents()
    s = bdm.Simulation(R=12.0, capacity=len(x), precision="fp32")
    s.set_agents(_as(mem, x), _as(mem, y), _as(mem, z), _as(mem, d), step=step)
    a = s.get_agents()
    assert a["step"] == step and a["n"] == len(x)
    # the buffer of this parity holds the input bit for bit (for step 1 it is
    # the device-side copy)
    assert np.array_equal(a["x"], x) and np.array_equal(a["y"], y) and np.array_equal(a["z"], z)
    assert np.array_equal(a["diam"], np.asarray(d, np.float32).astype(np.float64))
    s.step(2)  # both parities are read by the iterations
    assert s.get_agents()["n"] == len(x)
    s.close()


BAD = {
    "x nan": ("x", np.nan), "z inf": ("z", np.inf), "y -inf": ("y", -np.inf), "x 1e9": ("x", 1e9),
    "y -1e9": ("y", -1e9), "diam 0": ("d", 0.0), "diam negative": ("d", -5.0), "diam nan": ("d", np.nan),
    "diam inf": ("d", np.inf), "diam 1e6": ("d", 1e6),
}


@pytest.mark.parametrize("mem", ["host", "device"])
@pytest.mark.parametrize("kind", sorted(BAD))
def test_invalid_inputs_refused(mem, kind):
    x, y, z, d = _agents()
    arr = {"x": x, "y": y, "z": z, "d": d}
    name, v = BAD[kind]
    arr[name][1234] = v
    s = bdm.Simulation(R=12.0, capacity=len(x), precision="fp32")
    with pytest.raises(bdm.BdmError) as e:
        s.set_agents(_as(mem, x), _as(mem, y), _as(mem, z), _as(mem, d))
    assert e.value.code == bdm.BDM_EINVAL
    with pytest.raises(bdm.BdmError) as e:
        s.step(1)
    assert e.value.code == bdm.BDM_ESTATE
    # a valid set afterwards works
    x2, y2, z2, d2 = _agents(seed=6)
    s.set_agents(_as(mem, x2), _as(mem, y2), _as(mem, z2), _as(mem, d2))
    s.step(1)
    assert s.get_agents()["n"] == len(x2)
    s.close()
