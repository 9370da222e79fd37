"""Helpers for the GPU parity tests (imported by tests, not collected)."""
import numpy as np

MARGIN = 1e-5      # decisions whose oracle margin is below this are not compared bit for bit
FLOAT_RTOL = 1e-4  # FP32 state vs FP64 oracle, relative to the scale of the quantity


def torch_cuda():
    import torch
    return torch


def dev(a, dtype=None):
    import torch
    t = torch.from_numpy(np.ascontiguousarray(a))
    if dtype is not None:
        t = t.to(dtype)
    return t.cuda()


def host(t):
    import torch
    torch.cuda.synchronize()
    return t.cpu().numpy()


def compare_decisions(choice, step, ref, label=""):
    """Bit-exact choice and step wherever the oracle margin is >= MARGIN.
    Returns the number of excluded trials."""
    keep = ref["margin"] >= MARGIN
    bad_c = np.nonzero(keep & (choice != ref["choice"]))[0]
    bad_s = np.nonzero(keep & (step != ref["step"]))[0]
    assert bad_c.size == 0, (label, "choice mismatch", bad_c[:10], choice[bad_c[:10]],
                             ref["choice"][bad_c[:10]], ref["margin"][bad_c[:10]])
    assert bad_s.size == 0, (label, "step mismatch", bad_s[:10], step[bad_s[:10]],
                             ref["step"][bad_s[:10]], ref["margin"][bad_s[:10]])
    return int((~keep).sum())


def rel_err(gpu, ref, scale):
    """max |gpu - ref| / max(|ref|, scale) over elements."""
    gpu = np.asarray(gpu, np.float64)
    ref = np.asarray(ref, np.float64)
    den = np.maximum(np.abs(ref), scale)
    return float(np.max(np.abs(gpu - ref) / den)) if gpu.size else 0.0
