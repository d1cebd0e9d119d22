"""The metal-matrix composite's parameters used by the tests and the bench
(synth.ALUMINIUM_MS, synth.ALUMINA, in GPa and 1/s) are the paper's table
(tests/golden/misu_parameters.txt: Sec. 3, Table misu_parameters)."""
import os

import synth

UNIT = {"GPa": 1.0, "MPa": 1e-3, "1": 1.0, "1/s": 1.0}


def table():
    out = {}
    with open(os.path.join(os.path.dirname(__file__), "golden", "misu_parameters.txt")) as fh:
        for line in fh:
            if line.startswith("#") or not line.strip():
                continue
            phase, name, value, unit = line.split()
            out[(phase, name)] = float(value) * UNIT[unit]
    return out


def test_aluminium_matrix_is_the_papers():
    t = table()
    E, nu, sigY, H, edot0, sigd, n = synth.ALUMINIUM_MS
    assert (E, nu) == (t[("aluminium", "E")], t[("aluminium", "nu")])
    assert abs(sigY - t[("aluminium", "sigma_Y")]) < 1e-15 and abs(sigd - t[("aluminium", "sigma_d")]) < 1e-15
    assert (H, edot0, n) == (t[("aluminium", "H")], t[("aluminium", "edot0")], t[("aluminium", "n")])


def test_alumina_is_the_papers():
    t = table()
    assert tuple(synth.ALUMINA) == (t[("alumina", "E")], t[("alumina", "nu")])
