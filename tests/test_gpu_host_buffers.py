"""zbus_solve on host buffers: chunked staging with copies overlapping the
sweeps must give the same results, bit for bit, as the solve on device
buffers (every scenario's arithmetic is independent of its batch), for the
plain method and the defect forms, with and without a warm start, in one
chunk and in four."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

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


@pytest.mark.parametrize("mode", ["fp64", "fp16_scaled", "tree"])
@pytest.mark.parametrize("pinned", [True, False])
def test_host_buffers_equal_device_buffers(mode, pinned):
    f, Sw, Sd, w = F.make_workload("feeder128_b4096", B=3000)   # one chunk (36 MB of loads)
    net = zbus.Network.from_feeder(f)
    Vd, itd, cvd = net.solve(torch.from_numpy(Sw).cuda(), torch.from_numpy(Sd).cuda(),
                             precision=mode)
    hs = [torch.from_numpy(Sw), torch.from_numpy(Sd)]
    if pinned:
        hs = [x.pin_memory() for x in hs]
    Vh, ith, cvh = net.solve(hs[0], hs[1], precision=mode)
    torch.cuda.synchronize()
    assert not Vh.is_cuda
    assert torch.equal(Vh, Vd.cpu())
    assert torch.equal(ith, itd.cpu()) and torch.equal(cvh, cvd.cpu())
    # a warm start from the result: one sweep each
    V0 = Vh.clone()
    V2, it2, cv2 = net.solve(hs[0], hs[1], V_init=V0, precision=mode)
    torch.cuda.synchronize()
    Vd2, itd2, _ = net.solve(torch.from_numpy(Sw).cuda(), torch.from_numpy(Sd).cuda(),
                             V_init=Vd, precision=mode)
    assert torch.equal(V2, Vd2.cpu()) and torch.equal(it2, itd2.cpu())


@pytest.mark.parametrize("mode", ["fp16_scaled", "tree"])
def test_host_buffers_in_chunks_equal_device_buffers(mode):
    """Loads above 256 MB go through the device in four chunks (1/8, 3/8, 3/8
    and 1/8 of the batch, here 768, 2304, 2304 and 624 scenarios)."""
    f, Sw, Sd, w = F.make_workload("feeder1024_b16384", B=6000)   # 589 MB of loads
    net = zbus.Network.from_feeder(f)
    Vd, itd, cvd = net.solve(torch.from_numpy(Sw).cuda(), torch.from_numpy(Sd).cuda(),
                             precision=mode)
    for pinned in (True, False):
        hs = [torch.from_numpy(Sw), torch.from_numpy(Sd)]
        if pinned:
            hs = [x.pin_memory() for x in hs]
        Vh, ith, cvh = net.solve(hs[0], hs[1], precision=mode)
        torch.cuda.synchronize()
        assert torch.equal(Vh, Vd.cpu())
        assert torch.equal(ith, itd.cpu()) and torch.equal(cvh, cvd.cpu())
    assert cvd.all()
    net.close()


def test_mixed_buffer_kinds_are_refused():
    f, Sw, Sd, w = F.make_workload("feeder13_b8")
    net = zbus.Network.from_feeder(f)
    with pytest.raises(zbus.ZbusError):
        net.solve(torch.from_numpy(Sw), torch.from_numpy(Sd).cuda())
