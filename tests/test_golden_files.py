"""The stored expected values under tests/golden/ are the paper's (cited in
each file) or were written by a committed script that calls only oracle/;
the latter record the oracle source they were made with, which must be the
current one (CPU only)."""
import hashlib
import json
import os

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)


import pytest


@pytest.mark.parametrize("case,cells,n", [("sputter256", 256, 100_000), ("ccp128", 128, 20_000)])
def test_steady_state_reference_was_written_by_the_current_oracle(case, cells, n):
    with open(os.path.join(HERE, "golden", f"steady_state_{case}.json")) as fh:
        ref = json.load(fh)
    with open(os.path.join(ROOT, "oracle", "pic_oracle.c"), "rb") as fh:
        assert ref["oracle_sha16"] == hashlib.sha256(fh.read()).hexdigest()[:16], \
            "oracle changed: rerun tests/golden/make_steady_state_ref.py"
    assert len(ref["seeds"]) >= 8 and ref["n_cells"] == cells and ref["n_per_species"] == n
    for k in ("phi", "n_e", "n_i", "gamma_i"):
        assert len(ref["profiles"][k]["mean"]) == cells + 1
    for k in ("iedf_l", "iedf_r", "eedf"):
        assert ref["hists"][k]["pair_D_mean"] > 0
