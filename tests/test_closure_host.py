"""Host logic of the closure driver (paper_2504_08157_gb300/closure.py) that
needs no GPU: the choice of the output gain, with the plain right-hand side
(gain 0) as fallback."""


def test_gain_selection_falls_back_to_the_plain_rhs(monkeypatch):
    """select_gain scores each gain by its mean error relative to the plain
    run's (gain 0) and keeps the lowest: a closure that only hurts selects
    0, one that helps is selected, ties go to the smaller gain."""
    from paper_2504_08157_gb300 import closure as CL
    table = {}
    monkeypatch.setattr(CL, "evaluate_gains", lambda *a, **k: dict(table))
    plain = [0.02, 0.07, 0.07, 0.002, 0.02]
    table.update({0.0: plain, 0.1: [2 * e for e in plain], 1.0: [10 * e for e in plain]})
    assert CL.select_gain(None, 0, None, None, 0, None, gains=(0.0, 0.1, 1.0))[0] == 0.0
    table[0.1] = [0.5 * e for e in plain]
    assert CL.select_gain(None, 0, None, None, 0, None, gains=(0.0, 0.1, 1.0))[0] == 0.1
    table[1.0] = [0.5 * e for e in plain]
    assert CL.select_gain(None, 0, None, None, 0, None, gains=(0.0, 0.1, 1.0))[0] == 0.1
