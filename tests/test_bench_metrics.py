"""Host-side bookkeeping of bench.py: the paper's trace error (Section 3's
accuracy comparison), the tensor-core operation count and the algorithmic HBM
bytes of one step, each against a value fixed by its definition."""
import numpy as np
import pytest

import bench


def test_paper_err_closed_forms():
    rng = np.random.default_rng(0)
    ref = rng.normal(size=(200, 5, 3))
    assert bench.paper_err(ref, ref) == 0.0
    # a uniform relative gain eps on every channel: Err = eps^2 exactly
    for eps in (1e-3, -0.25):
        assert bench.paper_err(ref * (1.0 + eps), ref) == pytest.approx(eps * eps, rel=1e-12)
    # one channel off by its own amplitude, the others exact: Err = 1 / channels
    obs = ref.copy()
    obs[:, 2, 1] = 0.0
    assert bench.paper_err(obs, ref) == pytest.approx(1.0 / 15, rel=1e-12)


def test_paper_err_is_per_channel_not_pooled():
    """Channels are normalised by their own energy: a channel 100x weaker with
    the same relative error weighs as much as a strong one."""
    t = np.linspace(0, 1, 400)
    ref = np.stack([np.sin(9 * t), 0.01 * np.cos(5 * t)], axis=1)
    obs = ref.copy()
    obs[:, 1] *= 1.1   # 10 % error on the weak channel only
    assert bench.paper_err(obs, ref) == pytest.approx(0.5 * 0.01, rel=1e-12)
    pooled = np.sum((obs - ref) ** 2) / np.sum(ref ** 2)
    assert pooled < 1e-5


def test_paper_err_skips_silent_channels():
    ref = np.zeros((10, 2, 3))
    assert bench.paper_err(ref + 1.0, ref) is None
    ref[:, 0, 0] = 1.0
    obs = ref.copy()
    obs[:, 1, 2] = 5.0   # noise on a silent channel is not counted
    assert bench.paper_err(obs, ref) == 0.0


def test_tc_ops_per_element():
    # per stage: a 48 x 32 product (24 data + 8 bias columns) of multiply-adds
    assert bench.tc_ops_per_element(1) == 2 * 48 * 32
    assert bench.tc_ops_per_element(5) == 15360


def test_algorithmic_bytes():
    mesh = {"shape": (2, 3, 4)}
    nodes, elems = 3 * 4 * 5, 2 * 3 * 4
    assert bench.algorithmic_bytes_per_step(mesh) == 80 * nodes + 4 * elems
    assert bench.algorithmic_bytes_per_step(mesh, damped=True) == 128 * nodes + 4 * elems


def test_paper_err_leaves_out_channels_the_wave_has_not_reached():
    t = np.linspace(0, 1, 300)
    ref = np.stack([np.sin(7 * t), 1e-12 * np.sin(3 * t)], axis=1)
    obs = ref.copy()
    obs[:, 0] *= 1.0 + 1e-4
    obs[:, 1] = 0.0   # below the recorder's quantum: recorded as zero
    assert bench.paper_err(obs, ref) == pytest.approx(0.5 * (1e-8 + 1.0), rel=1e-6)
    err, n = bench.paper_err(obs, ref, rel_floor=1e-6, return_channels=True)
    assert n == 1
    assert err == pytest.approx(1e-8, rel=1e-6)
