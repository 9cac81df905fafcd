"""The JSON-lines metrics log of the binding (host logic, no GPU): every
record is one parseable line with its record type and time, appended to a
path or written to an open file."""
import io
import json

from paper_1007_3432_gb300.binding import MetricsLog


def test_records_are_json_lines(tmp_path):
    path = tmp_path / "m.jsonl"
    log = MetricsLog(str(path))
    log.write("solve", iterations=12, true_relres=9.5e-11, converged=1, d=3)
    log.write("result", ticket=4, kind=1, status=0, latency_ms=12.5, queued=3, active=7)
    log.close()
    lines = path.read_text().splitlines()
    assert len(lines) == 2
    a, b = (json.loads(l) for l in lines)
    assert a["record"] == "solve" and a["iterations"] == 12 and a["true_relres"] == 9.5e-11 and a["time"] > 0
    assert b["record"] == "result" and b["kind"] == 1 and b["queued"] == 3 and b["active"] == 7
    # appends to an existing path
    log2 = MetricsLog(str(path))
    log2.write("trajectory", dH=0.25, accepted=1)
    log2.close()
    assert len(path.read_text().splitlines()) == 3


def test_open_file_target_is_not_closed():
    buf = io.StringIO()
    log = MetricsLog(buf)
    log.write("action", S=1.5)
    log.close()
    assert not buf.closed
    assert json.loads(buf.getvalue())["S"] == 1.5
