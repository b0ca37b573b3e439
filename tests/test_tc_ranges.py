"""The K runs of the tensor-core contractions, checked on the host (no GPU): the library builds
each scale's runs as a plan does and checks them against the engines' tile rules
(crv_debug_check_tc_ranges). Every analysis tile with work must stay inside the runs its
operand tables were filled for (a chunk outside them would be read from memory no fill wrote)
and cover every l from the kernel's support on that its products need; every synthesis tile
whose output the reduction over m' reads must have work covering its n. Cases: the band limits
of the benchmark's scales with their support starts (first l with kappa^(j)(l) > 0 for
lambda = 2: lambda^(j-1) + 1), odd and ragged band limits, supports starting just below the
band limit, an empty support, all three column sets. A mismatch planted in the arguments (A
runs starting later than the B runs) must be caught."""
import pytest

import paper_1511_05578_gb300 as crv


def _lib_or_skip():
    try:
        crv.load()
    except Exception as e:  # pragma: no cover - the library is built by the ABI tests' fixture
        pytest.skip(f"library not loadable: {e}")


@pytest.fixture(scope="module", autouse=True)
def _built():
    import __graft_entry__ as g
    g.build()
    _lib_or_skip()


SCALES = [(8, 3), (16, 5), (32, 9), (64, 17), (128, 33), (256, 65), (512, 129), (512, 257), (1024, 257),
          (1024, 513)]
RAGGED = [(45, 12), (45, 0), (100, 37), (1000, 900), (1000, 999), (1000, 1000), (17, 16), (1, 0), (2, 1)]
KINDS = [(True, 0, False), (False, 2, False), (False, 0, True)]  # real spin 0; complex spin 2; unrotated


@pytest.mark.parametrize("Lb,lmin", SCALES + RAGGED)
@pytest.mark.parametrize("real,spin,unrot", KINDS)
def test_runs_follow_the_tile_rules(Lb, lmin, real, spin, unrot):
    bad, tiles = crv.crv_debug_check_tc_ranges(Lb, lmin, lmin, real, spin, unrot)
    assert tiles > 0
    assert bad == 0, (Lb, lmin, bad, tiles)


@pytest.mark.parametrize("Lb,lmin", [(1024, 0), (512, 0), (45, 0)])
def test_runs_from_max_mprime_n_as_before_the_support_start(Lb, lmin):
    assert crv.crv_debug_check_tc_ranges(Lb, lmin, lmin, True)[0] == 0


@pytest.mark.parametrize("Lb,lmin_b,lmin_a", [(1024, 513, 600), (256, 65, 100), (45, 0, 20)])
def test_a_runs_starting_after_the_b_runs_are_caught(Lb, lmin_b, lmin_a):
    bad, tiles = crv.crv_debug_check_tc_ranges(Lb, lmin_b, lmin_a, True)
    assert bad > 0, (Lb, lmin_b, lmin_a)


def test_a_runs_starting_earlier_are_harmless():
    assert crv.crv_debug_check_tc_ranges(1024, 513, 257, True)[0] == 0


@pytest.mark.parametrize("args", [(0, 0, 0, True), (1025, 0, 0, True), (64, -1, 0, True), (64, 65, 0, True),
                                  (64, 0, 65, True), (64, 0, 0, True, 2)])
def test_bad_arguments_are_rejected(args):
    with pytest.raises(crv.CrvError) as e:
        crv.crv_debug_check_tc_ranges(*args)
    assert e.value.status == crv.CRV_EINVAL
