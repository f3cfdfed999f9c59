"""What the trained closure gains over the method without it (GPU).

Training data come from the coupled method itself (channels of the
2048 x 512 family at Ny = 64 and 128, sampling only), the network is trained
by the library's own tcgen05 forward/backward kernels and Adam step, and the
test compares, on channels with other seeds and forces, the error of the
network's prediction and of the plain 8-frame mean -- the averaged coupling
restricted to the same 8 frames, hence the same lag -- against the same
target, the 500-step moving average of the strip fields."""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ct():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    import __graft_entry__
    __graft_entry__.build()
    from paper_2004_00304_gb300 import closure_train
    return closure_train


def test_trained_closure_beats_the_8_frame_mean(ct):
    train_ch = ct.training_channels(4, seed=1, ny_choices=(64, 128))
    test_ch = ct.training_channels(2, seed=2, ny_choices=(64, 128))
    X, T = ct.generate(train_ch, spinup=1500, samples=60, every=10)
    Xv, Tv = ct.generate(test_ch, spinup=1500, samples=20, every=25)
    theta, losses = ct.train(X, T, steps=1500, batch=32, lr=1e-3, seed=0)
    ev = ct.evaluate(theta, Xv, Tv)
    print(f"{X.shape[0]} training patches, {Xv.shape[0]} held-out; loss {losses[:20].mean():.4f} -> "
          f"{losses[-100:].mean():.4f}; RMS error net {np.round(ev['rmse_net'], 4)}, "
          f"8-frame mean {np.round(ev['rmse_mean8'], 4)}, gain {np.round(ev['gain'], 2)}")
    assert losses[-100:].mean() < 0.5 * losses[:20].mean()
    assert np.all(ev["gain"] > 1.5), ev["gain"]
