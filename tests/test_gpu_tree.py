"""Tree-sweep form on the GPU: radial structure detection and networks the
sweep inverts only in part.

The generic parity cases of the defect forms (against the FP64 oracle, one
step, full size, batch independence, zero load, divergence, the FP64
mismatch test) run the tree sweep through tests/test_gpu_mixed.py; batched
and served solves through tests/test_gpu_batched.py and tests/test_gpu_serve.py.
"""
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


def with_extra(f, extra):
    """COO of f's admittance plus extra entries {(row, col): value}."""
    row = list(f.Y_row) + [r for r, c in extra]
    col = list(f.Y_col) + [c for r, c in extra]
    val = list(f.Y_val) + list(extra.values())
    return (np.asarray(row, np.int32), np.asarray(col, np.int32),
            np.asarray(val, np.complex128))


def test_meshed_network_is_refused():
    f = F.make_feeder(20, 3, delta_frac=0.3)
    a, b = 5, 17
    y = np.linalg.inv(f.z_line[4])
    extra = {}
    for p in range(3):
        for q in range(3):
            extra[(3 * a + p, 3 * a + q)] = y[p, q]
            extra[(3 * b + p, 3 * b + q)] = extra.get((3 * b + p, 3 * b + q), 0) + y[p, q]
            extra[(3 * a + p, 3 * b + q)] = -y[p, q]
            extra[(3 * b + p, 3 * a + q)] = -y[p, q]
    row, col, val = with_extra(f, extra)
    net = zbus.Network(f.n_total, row, col, val, f.slack_idx, f.v_slack)
    Sw, Sd = F.make_scenarios(f, 4, 0.8, 1.2)
    with pytest.raises(zbus.ZbusError) as e:
        net.solve(dev(Sw), dev(Sd), precision="tree")
    assert "radial" in str(e.value)
    # the dense forms still solve it, and agree with the oracle
    Y = O.dense_from_coo(f.n_total, row, col, val)
    Y_LL, Y_Ls, _ = O.partition(Y, f.slack_idx)
    Z, w = O.reduced_impedance(Y_LL, Y_Ls, f.v_slack)
    ref, _, cv_ref = O.fixed_point(Z, w, Sw, Sd, 1e-8, 50)
    V, it, cv = net.solve(dev(Sw), dev(Sd), precision="fp16_scaled")
    assert (cv.cpu().numpy() == cv_ref).all()
    assert np.abs(V.cpu().numpy() - ref).max() <= 1e-6


@pytest.mark.parametrize("mode", ["tree", "fp16_scaled", "bf16x2"])
def test_shunts_converge_to_the_oracle(mode):
    # capacitive shunts: the sweep inverts only the series part, the defect
    # residual keeps them exactly (its shunt blocks, in the FP32 start sweeps
    # and in double-float); the dense forms invert them with Z
    f = F.make_feeder(90, 12, delta_frac=0.4)
    extra = {}
    for bus in (3, 9, 20, 33, 71):
        for p in range(3):
            extra[(3 * bus + p, 3 * bus + p)] = 0.02j
    row, col, val = with_extra(f, extra)
    net = zbus.Network(f.n_total, row, col, val, f.slack_idx, f.v_slack)
    Sw, Sd = F.make_scenarios(f, 70, 0.8, 1.2, seed=4)
    ref = O.solve_coo(f.n_total, row, col, val, f.slack_idx, f.v_slack, Sw, Sd)
    V, it, cv = net.solve(dev(Sw), dev(Sd), precision=mode)
    np.testing.assert_array_equal(cv.cpu().numpy(), ref["converged"])
    assert np.abs(V.cpu().numpy() - ref["V"]).max() <= 1e-6
    mm = net.power_mismatch(V, dev(Sw), dev(Sd)).cpu().numpy()
    assert mm.max() <= 1e-6


@pytest.mark.parametrize("N,B", [(2, 3), (13, 1), (256, 33), (1500, 6)])
def test_sizes_and_block_shapes(N, B):
    # one bus, a single scenario, a deep tree with few scenarios per block
    f = F.make_feeder(N, 40 + N, delta_frac=0.3)
    Sw, Sd = F.make_scenarios(f, B, 0.8, 1.2)
    ref = O.solve_coo(f.n_total, f.Y_row, f.Y_col, f.Y_val, f.slack_idx, f.v_slack, Sw, Sd)
    net = zbus.Network.from_feeder(f)
    V, it, cv = net.solve(dev(Sw), dev(Sd), precision="tree")
    np.testing.assert_array_equal(cv.cpu().numpy(), ref["converged"])
    m = ref["converged"] == 1
    assert np.abs(V.cpu().numpy()[m] - ref["V"][m]).max(initial=0.0) <= 1e-6
    assert np.abs(it.cpu().numpy()[m] - ref["iters"][m]).max(initial=0) <= 1


def test_tree_and_dense_forms_take_the_same_sweeps():
    f, Sw, Sd, w = F.make_workload("feeder128_b4096", B=512)
    net = zbus.Network.from_feeder(f)
    _, it64, _ = net.solve(dev(Sw), dev(Sd), precision="fp64")
    _, itt, cvt = net.solve(dev(Sw), dev(Sd), precision="tree")
    assert cvt.cpu().numpy().all()
    assert np.abs(itt.cpu().numpy() - it64.cpu().numpy()).max() <= 1
