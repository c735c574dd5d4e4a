"""Checkpoint files on the host: a cloud's snapshot survives a save / load round
trip unchanged, and restoring it into a cloud of another shape is refused."""
import pytest
import torch

from paper_2512_20829_gb300 import fla
from paper_2512_20829_gb300 import inputs as I


def test_cloud_snapshot_roundtrip_and_mismatch(tmp_path):
    wl = I.taylor_green_2d(scale=4)
    c = fla.DeviceCloud.from_seeds(wl.fla, 2, wl.delta, wl.dt, fla.F32X2, device="cpu")
    c.state.add_(torch.arange(c.state.numel(), dtype=c.state.dtype).reshape(c.state.shape) * 1e-3)
    c.meta.fill_(7)
    path = tmp_path / "c.pt"
    fla.save_checkpoint(path, {"step": 40, "fla": c.snapshot()})
    ck = fla.load_checkpoint(path, device="cpu")
    d = fla.DeviceCloud.from_seeds(wl.fla, 2, wl.delta, wl.dt, fla.F32X2, device="cpu")
    d.restore(ck["fla"])
    assert ck["step"] == 40
    assert torch.equal(d.state, c.state) and torch.equal(d.meta, c.meta)
    other = fla.DeviceCloud.from_seeds(I.taylor_green_2d(scale=2).fla, 2, wl.delta, wl.dt, fla.F32X2, device="cpu")
    with pytest.raises(fla.FlaError):
        other.restore(ck["fla"])
    folded = fla.DeviceCloud.from_seeds(wl.fla, 2, wl.delta, wl.dt, fla.F32, device="cpu")
    folded.state = folded.state.new_zeros(c.state.shape)
    folded.fold = torch.zeros(8, dtype=torch.float64)
    with pytest.raises(fla.FlaError):   # a snapshot without fold planes into a guarded cloud
        folded.restore(ck["fla"])
