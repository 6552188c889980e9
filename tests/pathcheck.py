"""Comparison of a GPU path (bl_fit_path-shaped dict) with an oracle path."""
import numpy as np

from paper_1701_05936_gb300 import bl


def compare_paths(prob, g, o, tol, obj_rtol=1e-7, allow_exempt=0):
    p = prob.p
    K = len(o["lambdas"])
    np.testing.assert_allclose(g["lambdas"].cpu().numpy(), o["lambdas"], rtol=2e-6 if prob.dtype == "f32" else 1e-12)
    B = bl.path_dense(g, p).cpu().numpy()
    Bo = o["beta"]
    diff = np.abs(B - Bo).max()
    assert diff <= tol, f"max |beta_gpu - beta_oracle| = {diff}"
    mism = (B != 0) != (Bo != 0)
    # an exemption: a feature entering exactly at this lambda (|beta| below tol on both sides)
    exempt = mism & (np.maximum(np.abs(B), np.abs(Bo)) < tol)
    assert np.sum(mism & ~exempt) == 0
    assert np.sum(exempt) <= allow_exempt, f"{np.sum(exempt)} near-tie active-set differences"
    loss = g["loss"].cpu().numpy()
    np.testing.assert_allclose(loss, o["loss"], rtol=obj_rtol)
    Bog = bl.path_dense(g, p, "val_orig").cpu().numpy()
    np.testing.assert_allclose(Bog, o["beta_orig"], atol=tol * 10 / max(1e-3, o["s"][o["keep"] > 0].min()))
    cs = np.abs(o["c"]) / np.where(o["s"] > 0, o["s"], 1.0)
    np.testing.assert_allclose(g["intercept"].cpu().numpy(), o["intercept"], atol=tol * (1 + cs.max() * p))
    assert g["n_active"].numpy().tolist() == [int(v) for v in (B != 0).sum(axis=1)]
    assert g["nnz"] == int((B != 0).sum())
    return diff
