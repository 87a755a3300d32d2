"""Host-side parts of the quench driver (no GPU): the seed summary and the argument checks."""
import json

import numpy as np
import pytest

from paper_1204_2088_gb300 import quench


def _rec(seed, hydro, ts, time, F, S, seg=0.1):
    return {"system": "A8B8", "grid": 48, "hydro": hydro, "seed": seed, "omega": 0.0, "tau_s": ts, "tau_b": 1.0,
            "step": int(time * 10), "time": time, "F": F, "S": S, "segregation": seg}


def test_summary_over_seeds():
    recs = [_rec(1, 1, 0.6, 200.0, 0.2415, 0.410), _rec(2, 1, 0.6, 200.0, 0.2417, 0.412),
            _rec(3, 1, 0.6, 200.0, 0.2416, 0.408), _rec(1, 0, 1.0, 200.0, 0.2422, 0.398),
            _rec(2, 0, 1.0, 200.0, 0.2421, 0.397), {"system": "A8B8", "grid": 48, "hydro": 0, "seed": 3, "step": 2000,
                                                   "error": "DSCF_ERR_NUMERIC"}]
    rows = quench.summarize(recs)
    assert [(r["hydro"], r["seeds"]) for r in rows] == [(0, 2), (1, 3)]
    hyd = rows[1]
    assert hyd["S"] == pytest.approx(0.410) and hyd["S_std"] == pytest.approx(np.std([0.410, 0.412, 0.408], ddof=1))
    assert rows[0]["F"] == pytest.approx(0.24215) and rows[0]["F_std"] > 0


def test_summarize_cli_and_argument_checks(tmp_path, capsys):
    f = tmp_path / "run.jsonl"
    f.write_text("\n".join(json.dumps(_rec(s, 1, 1.0, 100.0, 0.24 + s * 1e-4, 0.34)) for s in (1, 2)) + "\n")
    assert quench.main(["--summarize", str(f)]) == 0
    row = json.loads(capsys.readouterr().out.strip())
    assert row["seeds"] == 2 and row["S_std"] == 0.0
    with pytest.raises(SystemExit):
        quench.main(["--batch", "--viscosities", "1.0"])   # pairs only; refused before any device work
