"""The mutation table of `tests/oracle_mutants.py` stays in step with the oracle's source, and its
runner catches a mutant end to end (the full run is a manual command, about a minute per mutant)."""
import oracle_mutants as om


def test_every_mutation_site_occurs_exactly_once():
    src = open(om.SOURCE).read()
    names = [n for n, _, _ in om.MUTANTS]
    assert len(names) == len(set(names))
    for n, a, b in om.MUTANTS:
        assert a != b, n
        assert src.count(a) == 1, (n, src.count(a))


def test_runner_catches_a_total_strain_friction_trial():
    """The friction trial taken from the total strain instead of the increment (App. A.3) passes every
    closed-form pin of the law; the law invariants catch it."""
    caught, first = om.run_one("shear_total_not_incremental")
    assert caught, first
    assert "tests/test_oracle_invariants.py::" in first, first
