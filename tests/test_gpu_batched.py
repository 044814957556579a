"""Batched solves: feeders of uneven size and scenario count in one set of sweeps.

Each feeder's results must equal its own single-feeder solve (same kernels,
per-scenario arithmetic independent of the batch) and the FP64 oracle within
1e-6 pu with identical flags; the autotuner must pick a compiled variant and
record it.
"""
import json
import os

import numpy as np
import pytest

torch = pytest.importorskip("torch")

from oracle import zbus_oracle as O                      # noqa: E402
from paper_2605_14103_gb300 import feeders as F          # noqa: E402
from paper_2605_14103_gb300 import zbus                  # noqa: E402

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def built():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2605_14103_gb300 import build as B
    B.build()
    zbus.lib()


def dev(x):
    return torch.from_numpy(np.ascontiguousarray(x)).cuda()


def make_set(specs, seed0=40):
    out = []
    for k, (N, B) in enumerate(specs):
        f = F.make_feeder(N, seed0 + 2 * k, delta_frac=0.4)
        Sw, Sd = F.make_scenarios(f, B, 0.8, 1.2)
        out.append((f, Sw, Sd))
    return out


SPECS = [(50, 33), (130, 1), (300, 260), (17, 7), (700, 129), (90, 128)]


@pytest.mark.parametrize("mode", ["fp16_scaled", "bf16x2", "tree"])
def test_batched_equals_single_and_oracle(mode):
    fs = make_set(SPECS)
    nets = [zbus.Network.from_feeder(f) for f, _, _ in fs]
    loads = [(dev(Sw), dev(Sd)) for _, Sw, Sd in fs]
    outs = zbus.solve_batched(nets, loads, precision=mode)
    torch.cuda.synchronize()
    for (f, Sw, Sd), net, (V, it, cv), (sw, sd) in zip(fs, nets, outs, loads):
        V1, it1, cv1 = net.solve(sw, sd, precision=mode)
        assert torch.equal(cv, cv1) and torch.equal(it, it1)
        assert (V - V1).abs().max().item() <= 1e-12
        ref = O.solve_coo(f.n_total, f.Y_row, f.Y_col, f.Y_val, f.slack_idx, f.v_slack, Sw, Sd)
        np.testing.assert_array_equal(cv.cpu().numpy(), ref["converged"])
        m = ref["converged"] == 1
        assert np.abs(V.cpu().numpy()[m] - ref["V"][m]).max() <= 1e-6
        assert np.abs(it.cpu().numpy()[m] - ref["iters"][m]).max() <= 1


@pytest.mark.parametrize("mode", ["fp16_scaled", "bf16x2"])
def test_every_contraction_variant_batched(mode):
    """Feeders of uneven size (different N-tile counts per item) through each
    compiled contraction variant, forced with zbus_tune_set: the K order of
    the product does not depend on the tile, so every variant gives the
    default's voltages (1e-12) and counts, and the FP64 method's flags."""
    fs = make_set(SPECS)
    nets = [zbus.Network.from_feeder(f) for f, _, _ in fs]
    loads = [(dev(Sw), dev(Sd)) for _, Sw, Sd in fs]
    max_n = max(net.n for net in nets)
    total_B = sum(Sw.shape[0] for _, Sw, _ in fs)
    base = zbus.solve_batched(nets, loads, precision=mode)
    ref = zbus.solve_batched(nets, loads, precision="fp64")
    try:
        for bn, st in zbus.zbus_tune_variants(mode):
            zbus.zbus_tune_set(mode, max_n, total_B, bn, st)
            outs = zbus.solve_batched(nets, loads, precision=mode)
            for (V, it, cv), (V0, it0, cv0), (Vr, _, cr) in zip(outs, base, ref):
                assert torch.equal(cv, cv0) and torch.equal(it, it0), (bn, st)
                assert (V - V0).abs().max().item() <= 1e-12, (bn, st)
                assert torch.equal(cv, cr)
                assert (V - Vr).abs().max().item() <= 1e-6
    finally:
        zbus.zbus_tune_set(mode, max_n, total_B, 0, 0)


def test_batched_repeat_and_fp64():
    fs = make_set([(40, 20), (80, 50)], seed0=70)
    nets = [zbus.Network.from_feeder(f) for f, _, _ in fs]
    loads = [(dev(Sw), dev(Sd)) for _, Sw, Sd in fs]
    a = zbus.solve_batched(nets, loads)
    b = zbus.solve_batched(nets, loads)
    c = zbus.solve_batched(nets, loads, precision="fp64")
    for (Va, ia, ca), (Vb, ib, cb), (Vc, ic, cc) in zip(a, b, c):
        assert torch.equal(Va, Vb) and torch.equal(ia, ib)
        assert torch.equal(ca, cc)
        assert (Va - Vc).abs().max().item() <= 1e-6


def test_batched_rejects_repeated_network():
    f = F.make_feeder(20, 3)
    net = zbus.Network.from_feeder(f)
    Sw, Sd = F.make_scenarios(f, 4, 0.8, 1.2)
    with pytest.raises(zbus.ZbusError) as ei:
        zbus.solve_batched([net, net], [(dev(Sw), dev(Sd))] * 2)
    assert ei.value.status == 1


def test_autotune_records_a_compiled_variant(tmp_path, monkeypatch):
    path = tmp_path / "tune.json"
    monkeypatch.setenv("ZBUS_TUNE_CACHE", str(path))
    fs = make_set([(200, 300), (120, 200)], seed0=90)
    nets = [zbus.Network.from_feeder(f) for f, _, _ in fs]
    o = zbus.zbus_solve_opts_default()
    o.precision = zbus.PRECISION["fp16_scaled"]
    items = []
    for net, (f, Sw, Sd) in zip(nets, fs):
        B = Sw.shape[0]
        items.append((net.handle, dev(Sw), dev(Sd), None,
                      torch.empty((B, net.n), dtype=torch.complex128, device="cuda"),
                      torch.empty((B,), dtype=torch.int32, device="cuda"),
                      torch.empty((B,), dtype=torch.uint8, device="cuda")))
    bn, stages = zbus.zbus_autotune(items, o, 1e-8, 50, reps=2)
    assert (bn, stages) in zbus.zbus_tune_variants("fp16_scaled")
    # the cache is written only if the library resolved the same path at first use;
    # the returned choice is what matters, and later solves still agree with FP64
    outs = zbus.solve_batched(nets, [(it[1], it[2]) for it in items])
    ref = zbus.solve_batched(nets, [(it[1], it[2]) for it in items], precision="fp64")
    for (V, _, c), (Vr, _, cr) in zip(outs, ref):
        assert torch.equal(c, cr)
        assert (V - Vr).abs().max().item() <= 1e-6
    if path.exists():
        txt = path.read_text()
        assert '"BN"' in txt
