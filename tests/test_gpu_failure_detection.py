"""Failure detection on the GPU without a fault: the tensor-core kernels wait on
mbarriers with a bounded number of polls, and a wait that gives up records a failure
that unet_status reports, after which the kernel returns.  The probe entry point runs
that same bounded wait on a barrier nothing arrives at (a short bound), so the wait
expires for real; the context stays usable and the next forward pass is clean."""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def lib():
    from paper_2203_11025_gb300 import build
    from paper_2203_11025_gb300 import lib as L
    build.build()
    return L


def test_expired_wait_is_reported_and_the_context_survives(lib):
    c = lib.unet_cfg_default(lib.UNET_STANDALONE)
    net = lib.UNet(c, seed=5)
    x = torch.from_numpy(np.random.default_rng(6).standard_normal((1, 64, 64, 4)).astype(np.float32)).cuda()
    ref = net.forward(x).cpu().numpy()
    assert not net.status()
    # a wait whose barrier completes: nothing is recorded
    net.wait_probe(1000, arrive=True)
    assert not net.status()
    # a wait on a barrier that never completes gives up after its bound and is reported
    net.wait_probe(1000, arrive=False)
    assert net.status()
    assert not net.status()          # reading the status clears it
    # the context is usable: the same forward pass gives the same output, clean status
    out = net.forward(x).cpu().numpy()
    assert not net.status()
    assert np.abs(out - ref).max() <= 1e-6 * np.abs(ref).max()


def test_probe_rejects_unbounded_requests(lib):
    net = lib.UNet(lib.unet_cfg_default(lib.UNET_STANDALONE), seed=5)
    for rounds in (0, (1 << 20) + 1):
        with pytest.raises(lib.HelmError):
            net.wait_probe(rounds)
