"""The random-access probe (the roofline's denominators) in every swept shape.

Each (mode, accesses in flight, blocks per SM, threads) of the sweep must run
and report a positive time; shapes the probe is not compiled for must be
refused before any launch (HT_ERR_INVALID), and the rates must respect the
obvious ordering: a 64-byte read is not cheaper per access than a 32-byte one
by more than noise.
"""
import pytest

pytestmark = pytest.mark.gpu


def test_every_swept_shape_runs(cuda_lib):
    b = cuda_lib
    modes = tuple(range(13))
    rows = b.probe_sweep(gib=0.5, n_access=1 << 22, modes=modes, reps=1)
    want = sum(len(b.PROBE_SHAPES.get(m, b.DEFAULT_WRITE_SHAPES)) for m in modes)
    assert len(rows) == want
    assert all(r["per_s"] > 1e8 for r in rows), [r for r in rows if r["per_s"] <= 1e8]


def test_unsupported_shapes_are_refused(cuda_lib):
    import torch
    b = cuda_lib
    buf = torch.empty(64 << 20, dtype=torch.uint8, device="cuda")
    ptr = (buf.data_ptr() + 255) // 256 * 256
    n = (64 << 20) - 256
    for mode, inf, bps, thr in ((0, 32, 8, 256), (1, 16, 8, 256), (8, 128, 8, 256), (0, 8, 8, 512),
                                (0, 8, 65, 256), (0, 3, 8, 256), (13, 8, 8, 256), (0, 8, 8, 48),
                                (9, 32, 8, 256), (11, 16, 8, 256), (12, 32, 8, 256)):
        with pytest.raises(b.HtError):
            b.vss_probe_random_cfg(ptr, n, 1 << 16, mode, inf, bps, thr)
    # the default shape still answers through both entry points
    assert b.vss_probe_random(ptr, n, 1 << 20, 0) > 0
    assert b.vss_probe_random_cfg(ptr, n, 1 << 20, 0, 0, 0, 0) > 0


def test_plateau_rates_are_consistent(cuda_lib):
    b = cuda_lib
    r = b.random_access_rates(gib=2, n_access=1 << 24, modes=(0, 1, 8))
    # a 64-byte read moves two sectors: at most a little faster per access than
    # a 32-byte read, and a 4-byte read of a sector no slower than the full read
    assert r[1] <= 1.1 * r[0]
    assert r[8] >= 0.9 * r[0]
