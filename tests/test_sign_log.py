"""The per-step JSON-lines log of a sign-iteration report (host only, no GPU)."""
import json

from paper_2003_03868_gb300 import _ffi, write_sign_log


def test_log_has_one_record_per_step_and_a_summary(tmp_path):
    rep = _ffi.SignReport()
    rep.iterations, rep.converged, rep.fp64_from = 4, 1, 3
    for i, (r, nz) in enumerate([(0.5, 100), (0.2, 120), (1e-5, 130), (1e-10, 131)]):
        rep.residual_history[i] = r
        rep.nnzb_history[i] = nz
    rep.residual, rep.e_band, rep.flops = 1e-10, -3.5, 2e9
    path = tmp_path / "sign.jsonl"
    write_sign_log(rep, str(path))
    lines = [json.loads(line) for line in path.read_text().splitlines()]
    assert [d["step"] for d in lines[:-1]] == [1, 2, 3, 4]
    # the switch to FP64 at step 3: steps 1-2 in the low tier
    assert [d["tier"] for d in lines[:-1]] == ["bf16x3", "bf16x3", "fp64", "fp64"]
    assert [d["residual"] for d in lines[:-1]] == [0.5, 0.2, 1e-5, 1e-10]
    assert [d["nnzb_x"] for d in lines[:-1]] == [100, 120, 130, 131]
    s = lines[-1]
    assert s["summary"] and s["iterations"] == 4 and s["converged"] and s["e_band"] == -3.5


def test_fp64_run_logs_every_step_as_fp64(tmp_path):
    rep = _ffi.SignReport()
    rep.iterations, rep.fp64_from = 2, 1
    path = tmp_path / "s.jsonl"
    write_sign_log(rep, str(path))
    lines = [json.loads(line) for line in path.read_text().splitlines()]
    assert [d["tier"] for d in lines[:-1]] == ["fp64", "fp64"]
