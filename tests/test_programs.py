"""Host-side checks of the recurrence programs (no GPU): every class program
is generated and validated by the library (slots in range, no level writes a
slot that the same level reads), and its structure matches what the
Obara-Saika / Head-Gordon-Pople recurrences of the paper's "Computational
Details" fix in closed form."""
import pytest

from paper_2607_05622_gb300 import ltjk

MAXL = 3       # value classes: s, p, d, f
MAXL_GRAD = 2  # derivative classes: s, p, d


def ncart(l):
    return (l + 1) * (l + 2) // 2


def span(lo, hi):
    return sum(ncart(l) for l in range(max(lo, 0), hi + 1))


def classes(lmax=MAXL):
    for la in range(lmax + 1):
        for lb in range(la + 1):
            for lc in range(lmax + 1):
                for ld in range(lc + 1):
                    yield la, lb, lc, ld


@pytest.fixture(scope="module")
def L():
    from paper_2607_05622_gb300 import build
    build.build()
    ltjk.lib()
    return ltjk


@pytest.mark.parametrize("q", list(classes()))
def test_value_program_structure(L, q):
    la, lb, lc, ld = q
    p = L.class_program(la, lb, lc, ld, 0)
    assert p["ltot"] == la + lb + lc + ld
    # output tiles over ranges of a's components: the largest holds
    # ceil(na / tiles) of them; the light classes keep the whole block in one
    na, blk = ncart(la), ncart(lb) * ncart(lc) * ncart(ld)
    assert 1 <= p["tiles"] <= na
    assert p["outputs"] == -(-na // p["tiles"]) * blk
    if la + lb + lc + ld <= 6:
        assert p["tiles"] == 1
    # accumulators: [e0|f0] for l_a <= |e| <= l_a + l_b and l_c <= |f| <= l_c + l_d
    assert p["accumulators"] == span(la, la + lb) * span(lc, lc + ld)
    # every VRR level raises the total angular momentum by one
    assert p["vrr_levels"] == p["ltot"]
    # the horizontal program ends with one placement step per output; it needs
    # no recurrence steps beyond those exactly when b and d are both s shells
    assert p["hrr_steps"] >= p["outputs"]
    assert (p["hrr_steps"] == p["outputs"]) == (lb == 0 and ld == 0)
    # (ps|ss): one VRR step per Cartesian direction, 3 flops each
    if q == (1, 0, 0, 0):
        assert p["vrr_steps"] == 3 and p["vrr_flops"] == 9
    # the kernel's shared memory must fit one SM (227 KB for one CTA)
    assert max(p["smem_per_warp"]) <= 227 * 1024


@pytest.mark.parametrize("q", list(classes(MAXL_GRAD)))
def test_derivative_program_structure(L, q):
    la, lb, lc, ld = q
    p = L.class_program(la, lb, lc, ld, 1)
    assert p["ltot"] == la + lb + lc + ld + 1
    # nine output tiles: centres A, B, C x directions x, y, z (D by translational invariance)
    assert p["tiles"] == 9 and p["outputs"] == ncart(la) * ncart(lb) * ncart(lc) * ncart(ld)
    # channels: lowered (a-1 / b-1 / c-1 rectangle), raised a, raised b, raised c
    acc = (span(la - 1, la + lb) * span(lc - 1, lc + ld) + span(la + 1, la + lb + 1) * span(lc, lc + ld)
           + span(la, la + lb + 1) * span(lc, lc + ld) + span(la, la + lb) * span(lc + 1, lc + ld + 1))
    assert p["accumulators"] == acc
    assert max(p["smem_per_warp"]) <= 227 * 1024


def test_symmetric_lookup_and_errors(L):
    assert L.class_program(0, 1, 0, 0) == L.class_program(1, 0, 0, 0)
    with pytest.raises(L.LtjkError) as e:
        L.class_program(MAXL + 1, 0, 0, 0)
    assert e.value.code == L.EUNSUPPORTED
    with pytest.raises(L.LtjkError):
        L.class_program(0, 0, 0, 0, 2)
    # derivative programs stop at d: an f shell's would need g recurrences
    with pytest.raises(L.LtjkError) as e:
        L.class_program(MAXL_GRAD + 1, 0, 0, 0, 1)
    assert e.value.code == L.EUNSUPPORTED


def test_f_classes_are_tiled_to_fit(L):
    # (ff|ff): 10000 integrals; untiled its horizontal region alone is 35101
    # slots (274 KB at 8 bytes), beyond one CTA's shared memory
    p = L.class_program(3, 3, 3, 3)
    assert p["tiles"] > 1
    assert p["hrr_slots"] <= p["vrr_slots"]
    assert max(p["smem_per_warp"]) <= 227 * 1024
    assert p["accumulators"] == span(3, 6) ** 2
