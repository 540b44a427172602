"""Surrogate network kernels (forward, every gradient, Adam) against the FP64
oracle of oracle/mlp.py (needs a GB300).  FP32 arithmetic: outputs and
gradients within 2e-4 relative of the oracle (norm-wise per array)."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

from oracle import mlp as omlp  # noqa: E402
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


def init(rng, nin, nh, nout):
    return [rng.normal(size=(nh, nin)) / np.sqrt(nin), rng.normal(size=nh) * 0.1,
            rng.normal(size=(nh, nh)) / np.sqrt(nh), rng.normal(size=nh) * 0.1,
            rng.normal(size=(nout, nh)) / np.sqrt(nh), rng.normal(size=nout) * 0.1]


def flat(P):
    return np.concatenate([p.reshape(-1) for p in P]).astype(np.float32)


def unflat(v, nin, nh, nout):
    shapes = [(nh, nin), (nh,), (nh, nh), (nh,), (nout, nh), (nout,)]
    out, k = [], 0
    for sh in shapes:
        n = int(np.prod(sh))
        out.append(v[k:k + n].reshape(sh))
        k += n
    return out


def rel(a, b):
    return np.linalg.norm(np.asarray(a, float) - b) / np.linalg.norm(b)


@pytest.mark.parametrize("dims,batch", [((4, 256, 1024), 256), ((4, 256, 1024), 37),
                                        ((3, 70, 100), 129)])
def test_mlp_forward_and_gradients(dims, batch):
    nin, nh, nout = dims
    rng = np.random.default_rng(batch)
    P = init(rng, nin, nh, nout)
    P32 = [p.astype(np.float32).astype(np.float64) for p in P]
    u = rng.uniform(-1, 1, (batch, nin)).astype(np.float32)
    t = rng.normal(size=(batch, nout)).astype(np.float32) * 0.1
    h = nb.nbody_mlp_create(nin, nh, nout, 256)
    assert nb.nbody_mlp_num_params(h) == sum(p.size for p in P)
    nb.nbody_mlp_set_params(h, torch.tensor(flat(P), device=DEV))
    U = torch.tensor(u, device=DEV)
    T = torch.tensor(t, device=DEV)
    Y = torch.empty((batch, nout), dtype=torch.float32, device=DEV)
    nb.nbody_mlp_forward(h, U, Y)
    y_ref, cache = omlp.forward(P32, u.astype(np.float64))
    assert rel(Y.cpu().numpy(), y_ref) <= 2e-5
    G = torch.empty(nb.nbody_mlp_num_params(h), dtype=torch.float32, device=DEV)
    DU = torch.empty((batch, nin), dtype=torch.float32, device=DEV)
    L = nb.nbody_mlp_loss_grad(h, U, T, G, DU)
    assert L == pytest.approx(omlp.mse(y_ref, t.astype(np.float64)), rel=1e-5)
    g_ref, du_ref = omlp.backward(P32, cache, y_ref, t.astype(np.float64))
    for got, ref in zip(unflat(G.cpu().numpy(), nin, nh, nout), g_ref):
        assert rel(got, ref) <= 2e-4
    assert rel(DU.cpu().numpy(), du_ref) <= 2e-4
    # two Adam steps against the oracle's update rule applied to the GPU's
    # own gradients (isolates the optimiser)
    w = flat(P).astype(np.float64)
    m = np.zeros_like(w)
    v = np.zeros_like(w)
    for step in (1, 2):
        g = np.empty(w.size, np.float32)
        Gs = torch.empty_like(G)
        nb.nbody_mlp_loss_grad(h, U, T, Gs, None, want_loss=False)
        g = Gs.cpu().numpy().astype(np.float64)
        nb.nbody_mlp_adam_step(h, 1e-3)
        w, m, v = omlp.adam_step(w, g, m, v, step, 1e-3)
        out = np.empty(w.size, np.float32)
        nb.nbody_mlp_get_params(h, out)
        assert np.abs(out - w).max() <= 1e-6 + 1e-5 * np.abs(w).max()
    nb.nbody_mlp_destroy(h)


def test_mlp_training_reduces_loss_reproducibly():
    rng = np.random.default_rng(3)
    nin, nh, nout, B = 4, 64, 16, 128
    u = rng.uniform(-1, 1, (B, nin)).astype(np.float32)
    t = np.sin(u @ rng.normal(size=(nin, nout))).astype(np.float32)
    runs = []
    for _ in range(2):
        h = nb.nbody_mlp_create(nin, nh, nout, B)
        nb.nbody_mlp_set_params(h, flat(init(np.random.default_rng(4), nin, nh, nout)))
        U, T = torch.tensor(u, device=DEV), torch.tensor(t, device=DEV)
        losses = []
        for it in range(300):
            losses.append(nb.nbody_mlp_loss_grad(h, U, T, want_loss=(it % 50 == 0 or it == 299)))
            nb.nbody_mlp_adam_step(h, 3e-3)
        out = np.empty(nb.nbody_mlp_num_params(h), np.float32)
        nb.nbody_mlp_get_params(h, out)
        runs.append(out)
        nb.nbody_mlp_destroy(h)
        assert losses[-1] < 0.05 * losses[0]
    assert np.array_equal(runs[0], runs[1])
