"""Failure detection of the surrogate network's tensor-core GEMM (needs a
GB300): its waits for the tensor cores are bounded.  With the test switch
NBODY_MLP_TEST_NO_MMA=1 at creation the GEMMs issue no MMA, so nothing
arrives on their mbarriers; every wait gives up after its bound (1 s of the
GPU's global timer), the status reads NBODY_ETIMEOUT, each block still frees
its tensor memory, and the GPU context stays usable: a network created
afterwards computes as before.  No trap, fault or unbounded wait."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

from paper_2511_22468_gb300 import nbody as nb  # noqa: E402

pytestmark = pytest.mark.gpu
DEV = torch.device("cuda:0")


@pytest.fixture(scope="module", autouse=True)
def _lib():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2511_22468_gb300 import build
    build.build()
    nb.lib()


def _forward(h, nin, nout, batch, seed):
    rng = np.random.default_rng(seed)
    u = torch.tensor(rng.uniform(-1, 1, (batch, nin)).astype(np.float32), device=DEV)
    y = torch.full((batch, nout), float("nan"), dtype=torch.float32, device=DEV)
    nb.nbody_mlp_forward(h, u, y)
    return y


def test_expired_tensor_core_wait_is_reported_and_the_context_survives(monkeypatch):
    nin, nh, nout, batch = 4, 64, 32, 8
    params = np.random.default_rng(1).normal(size=nin * nh + nh + nh * nh + nh + nout * nh + nout)
    params = torch.tensor((0.1 * params).astype(np.float32), device=DEV)

    monkeypatch.setenv("NBODY_MLP_TEST_NO_MMA", "1")
    h = nb.nbody_mlp_create(nin, nh, nout, batch)
    monkeypatch.delenv("NBODY_MLP_TEST_NO_MMA")
    nb.nbody_mlp_set_params(h, params)
    _forward(h, nin, nout, batch, 2)
    assert nb.nbody_mlp_get_status(h) == nb.NBODY_ETIMEOUT
    nb.nbody_mlp_destroy(h)
    torch.cuda.synchronize()

    # a network created without the switch: finite outputs, status OK, and
    # the same outputs as a second one (the tensor memory was released)
    outs = []
    for _ in range(2):
        g = nb.nbody_mlp_create(nin, nh, nout, batch)
        nb.nbody_mlp_set_params(g, params)
        y = _forward(g, nin, nout, batch, 2)
        assert nb.nbody_mlp_get_status(g) == nb.NBODY_OK
        outs.append(y.cpu().numpy())
        nb.nbody_mlp_destroy(g)
    assert np.all(np.isfinite(outs[0])) and np.array_equal(outs[0], outs[1])
