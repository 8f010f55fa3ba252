"""The 9-species input mechanism carries the reaction topology of the
paper's Appendix A (golden fixture tests/golden/appendix_a_h2air.txt)."""
import os

from paper_1110_4903_gb300 import synth

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "appendix_a_h2air.txt")


def _read_golden():
    out = []
    for line in open(GOLDEN):
        if line.startswith("#") or not line.strip():
            continue
        idx, re, pr, m = [p.strip() for p in line.split("|")]
        out.append((int(idx), tuple(sorted(re.split())), tuple(sorted(pr.split())), int(m)))
    return out


def _side(mech, sp, nu, r):
    names = []
    for j in range(3):
        if sp[r, j] >= 0:
            names += [mech.species[sp[r, j]]] * int(nu[r, j])
    return tuple(sorted(names))


def test_appendix_a_topology():
    gold = _read_golden()
    assert len(gold) == 19
    assert [g[0] for g in gold if g[3]] == [5, 6, 7, 8, 10, 15]
    mech = synth.h2_air_9sp()
    assert mech.ns == 9 and mech.nr == 38 and int(mech.third_body.sum()) == 6
    for r, (_, re, pr, m) in enumerate(gold):
        got = {_side(mech, mech.reac_sp, mech.reac_nu, r), _side(mech, mech.prod_sp, mech.prod_nu, r)}
        assert got == {re, pr}, r          # either orientation: reactions are reversible
        assert mech.third_body[r] == m


def test_paper_sized_mechanisms():
    m36 = synth.hydrocarbon_36sp()
    assert (m36.ns, m36.nr, m36.ne, int(m36.third_body.sum())) == (36, 308, 4, 40)
    for m in (synth.h2_air_9sp(), m36):
        assert (m.arr_A >= 1e8).all() and (m.arr_A <= 1e14).all()
        assert (abs(m.arr_beta) <= 1).all() and (m.arr_Ea >= 0).all() and (m.arr_Ea <= 2e5).all()
        assert (m.reac_nu.sum(1) <= 3).all() and (m.prod_nu.sum(1) <= 3).all()
        # reactions are distinct
        keys = {frozenset([_side(m, m.reac_sp, m.reac_nu, r), _side(m, m.prod_sp, m.prod_nu, r)])
                for r in range(m.nr)}
        assert len(keys) == m.nr
