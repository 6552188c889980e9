"""Comparison of a GPU path (bl_fit_path-shaped dict) with an oracle path."""
import numpy as np

from paper_1701_05936_gb300 import bl


def compare_paths(prob, g, o, tol, obj_rtol=1e-7, allow_exempt=0, label=""):
    """Assert the GPU path equals the oracle's within `tol` on the standardized
    coefficients, with identical active sets, and return
    (max |beta_gpu - beta_oracle|, number of exempted near-tie features).

    The one permitted active-set difference is a feature whose |beta| is below
    `tol` on both sides (a feature entering exactly at that lambda); the count
    of such exemptions is printed and must not exceed `allow_exempt`."""
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
    n_exempt = int(np.sum(exempt))
    print(f"compare_paths{(' ' + label) if label else ''}: K={K} max|dbeta|={diff:.3e} "
          f"active-set exemptions={n_exempt}")
    assert np.sum(mism & ~exempt) == 0
    assert n_exempt <= allow_exempt, f"{n_exempt} near-tie active-set differences"
    loss = g["loss"].cpu().numpy()
    np.testing.assert_allclose(loss, o["loss"], rtol=obj_rtol)
    Bog = bl.path_dense(g, p, "val_orig").cpu().numpy()
    np.testing.assert_allclose(Bog, o["beta_orig"], atol=tol * 10 / max(1e-3, o["s"][o["keep"] > 0].min()))
    # intercept_k = ybar - sum_j c_j beta_kj / s_j: its error is at most the sum, over
    # the features active on either side at lambda_k, of |c_j / s_j| |delta beta_kj|
    cs = np.abs(o["c"]) / np.where(o["s"] > 0, o["s"], 1.0)
    either = (B != 0) | (Bo != 0)
    atol_k = tol * (either * cs[None, :]).sum(axis=1) + 1e-9 * (1.0 + abs(o["ybar"]))
    ierr = np.abs(g["intercept"].cpu().numpy() - o["intercept"])
    assert np.all(ierr <= atol_k), f"intercept error {ierr.max():.3e} above its bound at lambda {int(np.argmax(ierr - atol_k))}"
    assert g["n_active"].numpy().tolist() == [int(v) for v in (B != 0).sum(axis=1)]
    assert g["nnz"] == int((B != 0).sum())
    return diff, n_exempt
