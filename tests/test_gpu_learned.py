"""The learned scatter estimator against the method without it.

Training pairs come from the method itself: seeded torsos at random gantry
angles, input = (Poisson-denoised 1e6-history MC scatter, ray-traced
primary), target = Poisson-denoised 1e8-history MC scatter.  The network is
trained on the GPU by the library's own forward, backward and Adam kernels.
On held-out torsos, against a 1e9-history denoised reference, it must beat
the plain method at the same photon count (denoised 1e6-history MC); the
relative l2 norm is the paper's scatter-image metric (Section 3.2).
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def gd():
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    from paper_1204_6367_gb300 import build, gdrr
    build.build()
    gdrr.lib()
    return gdrr


def test_network_beats_plain_method_at_equal_photons(gd):
    from paper_1204_6367_gb300 import scatter_net as sn
    X, Y = sn.make_dataset(range(100, 132), 4, 10**6, 10**8, rng_seed=1)
    net = gd.Cnn(16, sn.H, sn.W, 32, seed=1)
    losses = sn.train(net, X, Y, 1500, 16, 1e-3)
    assert np.mean(losses[-50:]) < 0.2 * np.mean(losses[:50])
    rng = np.random.default_rng(7)
    err_net, err_plain = [], []
    for s in (900, 901):
        with gd.Context(sn.coarse_problem(s)) as ctx:
            for a in range(2):
                ang = float(rng.uniform(0, 2 * np.pi))
                x = torch.empty((1, 2, sn.H, sn.W), dtype=torch.float32, device="cuda")
                d_low = sn.low_input(ctx, 10**6, 31 + 10 * s + a, ang, a, x[0]).cpu().numpy()
                ref = sn.estimate(ctx, 10**9, 91 + 10 * s + a, ang, a, 1.5)[0].cpu().numpy()
                pred = sn.predict(net, x).cpu().numpy()[0]
                err_net.append(sn.rel_l2(pred, ref))
                err_plain.append(sn.rel_l2(d_low, ref))
    print("learned vs plain (relative l2 against 1e9 reference):", np.mean(err_net), np.mean(err_plain))
    assert np.mean(err_net) < np.mean(err_plain), (err_net, err_plain)
    net.close()
