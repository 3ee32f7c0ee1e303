"""The sweep's command line (no GPU): every flag reaches run() as documented,
and each setting prints one JSON line."""
import json

from paper_1503_04500_gb300 import sweep


def test_command_line_reaches_run(monkeypatch, capsys):
    seen = {}

    def fake_run(workload, size, seed, eps, c, lmax, drop, tol, precision, side, rebuilds, solve, init, select,
                 A=None, global_ctas=0):
        seen.update(workload=workload, size=size, seed=seed, eps=eps, c=c, lmax=lmax, drop=drop, tol=tol,
                    precision=precision, side=side, rebuilds=rebuilds, solve=solve, init=init, select=select,
                    A=A, global_ctas=global_ctas)
        for e in eps:
            yield {"eps": e}

    monkeypatch.setattr(sweep, "run", fake_run)
    sweep.main(["--workload", "powerlaw", "--size", "5000", "--eps", "0.3,0.4", "--c", "5", "--lmax", "8",
                "--precision", "fp32_refine", "--rebuilds", "1", "--no-solve", "--global-ctas", "32",
                "--select", "spai", "--init", "A"])
    assert seen == dict(workload="powerlaw", size=5000, seed=1503, eps=[0.3, 0.4], c=[5], lmax=[8], drop="fixed",
                        tol=1e-3, precision="fp32_refine", side="right", rebuilds=1, solve=False, init="A",
                        select="spai", A=None, global_ctas=32)
    lines = capsys.readouterr().out.strip().splitlines()
    assert [json.loads(ln) for ln in lines] == [{"eps": 0.3}, {"eps": 0.4}]


def test_global_ctas_defaults_to_one_per_sm(monkeypatch):
    seen = {}

    def fake_run(workload, size, seed, eps, c, lmax, drop, tol, precision, side, rebuilds, solve, init, select,
                 A=None, global_ctas=-1):
        seen["global_ctas"] = global_ctas
        return iter(())

    monkeypatch.setattr(sweep, "run", fake_run)
    sweep.main(["--workload", "convdiff2d"])
    assert seen["global_ctas"] == 0
