import os
import sys

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA GPU (GB300, sm_103a)")
    config.addinivalue_line("markers", "slow: longer CPU test")


def has_gpu():
    try:
        import torch
        return torch.cuda.is_available()
    except Exception:
        return False


def pytest_collection_modifyitems(config, items):
    if has_gpu():
        return
    skip = pytest.mark.skip(reason="no CUDA GPU")
    for it in items:
        if "gpu" in it.keywords:
            it.add_marker(skip)


@pytest.fixture(scope="session")
def mechs():
    import synth
    cache = {}

    def get(name):
        if name not in cache:
            cache[name] = synth.make_mechanism(name)
        return cache[name]
    return get


def pytest_terminal_summary(terminalreporter):
    """How much the parity checks leaned on the oracle's rounding envelope:
    per check, the entries that passed only through the envelope (their
    error above rtol |ref| but within rtol env), and the well-conditioned
    entries (env <= 10 |ref|) that met the plain per-entry bar."""
    try:
        from tests.parity import REPORT, NEWTON_REPORT
    except Exception:
        return
    tr = terminalreporter
    if NEWTON_REPORT:
        tr.write_sep("-", "FP32 Newton matrix against the FP64 oracle")
        for r in NEWTON_REPORT:
            tr.write_line(f"  {r['what']}: {r['entries']} entries of {r['states']} states; |dM| / (|M| + h gamma "
                          f"env): median {r['entry_median']:.2e}, p99 {r['entry_p99']:.2e}, max "
                          f"{r['entry_max']:.2e}; ||dM||_F / ||M||_F median {r['frob_median']:.2e}, max "
                          f"{r['frob_max']:.2e}")
    if not REPORT:
        return
    ent = sum(r["entries"] for r in REPORT)
    env = sum(r["needed_env"] for r in REPORT)
    well = sum(r["well"] for r in REPORT)
    worst = max(r["worst_rel_well"] for r in REPORT)
    tr.write_sep("-", "parity checks against the oracle")
    tr.write_line(f"{len(REPORT)} checks, {ent} entries: {env} ({100.0 * env / max(ent, 1):.2f} %) passed only "
                  f"through the envelope; {well} ({100.0 * well / max(ent, 1):.2f} %) well-conditioned entries held "
                  f"to rtol |ref| (largest relative error {worst:.2e})")
    top = sorted(REPORT, key=lambda r: -r["needed_env"] / max(r["entries"], 1))[:12]
    for r in top:
        tr.write_line(f"  {r['needed_env']:>9} / {r['entries']:<9} via envelope, {r['well']:>9} well-conditioned "
                      f"(max rel {r['worst_rel_well']:.1e})  {r['what']}")
