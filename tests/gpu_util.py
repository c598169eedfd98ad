"""Helpers shared by the GPU tests: device upload, oracle comparison with the stated
tolerance (max relative error 1e-5 per non-zero entry of the FP64 oracle, exact zeros)."""
import numpy as np

RTOL = 1e-5


def dev_graph(g, device="cuda"):
    import torch
    t = lambda a: None if a is None else torch.from_numpy(np.ascontiguousarray(a)).to(device)
    return t(g.src), t(g.dst), t(g.w), t(g.labels)


def z_errors(Zg, Zo):
    """(max relative error over non-zero oracle entries, #entries non-zero on the GPU where
    the oracle is exactly zero)."""
    Zg = np.asarray(Zg, np.float64)
    nz = Zo != 0
    bad_zero = int(np.count_nonzero(Zg[~nz]))
    rel = np.abs(Zg[nz] - Zo[nz]) / np.abs(Zo[nz]) if nz.any() else np.zeros(1)
    return float(rel.max(initial=0.0)), bad_zero


def z_error_report(Zg, Zo, what):
    """One line with the max and 99th-percentile relative error over the non-zero oracle
    entries (shown by pytest -s)."""
    Zg = np.asarray(Zg, np.float64)
    nz = Zo != 0
    rel = np.abs(Zg[nz] - Zo[nz]) / np.abs(Zo[nz]) if nz.any() else np.zeros(1)
    line = (f"parity {what}: max relative error {rel.max(initial=0.0):.2e}, "
            f"p99 {np.percentile(rel, 99):.2e}, over {int(nz.sum())} non-zero entries")
    print(line)
    return line


def assert_z_matches(Zg, Zo, rtol=RTOL, what=""):
    err, bad = z_errors(Zg, Zo)
    assert bad == 0, f"{what}: {bad} entries non-zero where the oracle is zero"
    assert err <= rtol, f"{what}: max relative error {err:.3e} > {rtol:g}"
    return err
