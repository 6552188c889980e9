"""Proposer parameter files: bl_mlp_save / bl_mlp_load round-trip FP32 values
exactly and reject a file of the wrong shape (host only, no GPU)."""
import numpy as np
import torch

from paper_1701_05936_gb300 import bl


def test_mlp_save_load_roundtrip_and_rejects_bad_files(tmp_path):
    w = torch.from_numpy(np.random.default_rng(3).standard_normal(bl.BL_MLP_NPARAM).astype(np.float32))
    path = str(tmp_path / "proposer.txt")
    bl.mlp_save(w, path)
    assert torch.equal(bl.mlp_load(path), w)
    lines = open(path).read().splitlines()
    assert lines[0] == "biglasso-proposer 5 64 64 1" and len(lines) == 1 + bl.BL_MLP_NPARAM
    (tmp_path / "short.txt").write_text("\n".join(lines[:-1]) + "\n")
    (tmp_path / "wide.txt").write_text("biglasso-proposer 5 32 64 1\n" + "\n".join(lines[1:]) + "\n")
    for bad in ("short.txt", "wide.txt", "missing.txt"):
        try:
            bl.mlp_load(str(tmp_path / bad))
        except bl.BLError as e:
            assert e.status == bl.BL_ERR_ARG
        else:
            raise AssertionError(f"{bad} was accepted")
