"""Checkpoint files of a granule state (save_checkpoint / load_checkpoint):
host-side, no GPU needed.  A state round-trips bit for bit with its step and
metadata; files of another format or with inconsistent arrays are refused."""
import numpy as np
import pytest
import torch

from paper_2504_00745_gb300.gic import GIC_FP32, GIC_FP64, State
from paper_2504_00745_gb300.window import load_checkpoint, save_checkpoint


def random_state(n, prec, seed=0, with_posf=True):
    g = torch.Generator().manual_seed(seed)
    st = State.empty(n, prec, device="cpu", with_posf=with_posf)
    st.cell.copy_(torch.randint(0, 1 << 30, (n,), generator=g, dtype=torch.int32))
    if prec == GIC_FP32:
        st.pos.copy_(torch.randint(-(1 << 31), (1 << 31) - 1, (n, 4), generator=g, dtype=torch.int32))
    else:
        st.pos.copy_(torch.rand((n, 4), generator=g, dtype=torch.float64))
    st.vel.copy_(torch.randn((n, 4), generator=g, dtype=st.real))
    st.id.copy_(torch.randperm(n, generator=g).to(torch.int32))
    if st.posf is not None:
        st.posf.copy_(torch.randn((n, 4), generator=g, dtype=torch.float32))
    return st


@pytest.mark.parametrize("prec", [GIC_FP32, GIC_FP64])
def test_round_trip_is_exact(tmp_path, prec):
    st = random_state(1000, prec, with_posf=(prec == GIC_FP32))
    meta = {"workload": "dam_break_1m", "dt_sub": 2e-5, "sizes": [128, 128, 128]}
    path = tmp_path / "state.pt"
    save_checkpoint(path, st, step=4200, meta=meta)
    back, step, m = load_checkpoint(path, device="cpu")
    assert step == 4200 and m == meta and back.precision == prec
    for a, b in ((st.cell, back.cell), (st.pos, back.pos), (st.vel, back.vel), (st.id, back.id)):
        assert a.dtype == b.dtype and torch.equal(a, b)
    if prec == GIC_FP32:
        assert torch.equal(st.posf.view(torch.int32), back.posf.view(torch.int32))  # bits, NaN payloads included
    else:
        assert back.posf is None


def test_state_without_ids_and_empty_state(tmp_path):
    st = random_state(5, GIC_FP32, with_posf=False)
    st.id = None
    save_checkpoint(tmp_path / "a.pt", st)
    back, step, meta = load_checkpoint(tmp_path / "a.pt", device="cpu")
    assert back.id is None and back.posf is None and step == 0 and meta == {}
    empty = State.empty(0, GIC_FP64, device="cpu")
    save_checkpoint(tmp_path / "e.pt", empty)
    assert load_checkpoint(tmp_path / "e.pt", device="cpu")[0].n == 0


def test_foreign_or_inconsistent_files_are_refused(tmp_path):
    torch.save({"format": "something-else"}, tmp_path / "x.pt")
    with pytest.raises(ValueError, match="not a"):
        load_checkpoint(tmp_path / "x.pt", device="cpu")
    st = random_state(10, GIC_FP32)
    save_checkpoint(tmp_path / "s.pt", st)
    d = torch.load(tmp_path / "s.pt", weights_only=True)
    d["vel"] = d["vel"].double()  # an FP64 velocity in an FP32 state
    torch.save(d, tmp_path / "bad.pt")
    with pytest.raises(ValueError, match="do not form"):
        load_checkpoint(tmp_path / "bad.pt", device="cpu")
    d = torch.load(tmp_path / "s.pt", weights_only=True)
    d["pos"] = d["pos"][:5]
    torch.save(d, tmp_path / "short.pt")
    with pytest.raises(ValueError, match="do not form"):
        load_checkpoint(tmp_path / "short.pt", device="cpu")


def test_grid_is_recorded_and_checked(tmp_path):
    """Positions are contact-cell ids plus offsets in units of dx / k_contact:
    a state loaded on another grid would put every granule elsewhere, so a
    load that names a grid refuses a file from another one (or one that
    records none)."""
    from gic_inputs import Grid

    g = Grid(32, 32, 32, 1.0 / 32, k_contact=3)
    st = random_state(20, GIC_FP32)
    save_checkpoint(tmp_path / "g.pt", st, grid=g)
    back, _, _ = load_checkpoint(tmp_path / "g.pt", device="cpu", grid=g)
    assert torch.equal(back.pos, st.pos)
    for other in (Grid(32, 32, 32, 1.0 / 32, k_contact=2), Grid(32, 32, 16, 1.0 / 32, k_contact=3),
                  Grid(32, 32, 32, 1.0 / 64, k_contact=3), Grid(32, 32, 32, 1.0 / 32, origin=(0.5, 0, 0), k_contact=3)):
        with pytest.raises(ValueError, match="saved on grid"):
            load_checkpoint(tmp_path / "g.pt", device="cpu", grid=other)
    save_checkpoint(tmp_path / "nogrid.pt", st)
    with pytest.raises(ValueError, match="records no grid"):
        load_checkpoint(tmp_path / "nogrid.pt", device="cpu", grid=g)
    assert load_checkpoint(tmp_path / "nogrid.pt", device="cpu")[0].n == 20
