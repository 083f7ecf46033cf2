"""Host logic of the schedule autotuner: candidate lists and even row splits."""
from paper_0910_3915_gb300 import tune


def test_even_splits_fill_whole_waves():
    # 128^3 with 8-row tiles on 152 SMs x 2 CTAs: 19 tiles of 6-7 rows x 4 segments = 304 items
    assert (19, 4) in tune.even_splits(128, 128, 8, 304)
    for nx, ny, ty, ctas in ((128, 128, 8, 304), (256, 256, 8, 304), (128, 128, 4, 456), (37, 23, 8, 304)):
        ntx = -(-nx // 32)
        for nty, seg in tune.even_splits(nx, ny, ty, ctas):
            assert (ntx * nty * seg) % ctas == 0
            rows = -(-ny // nty)
            assert ty - 1 <= rows <= ty and nty <= ny


def test_candidates_and_names_round_trip():
    c = tune.candidates(126, "f32", nx=128, ny=128, n_sm=152)
    assert ("ldg", 0, 8, 4, 19) in c and ("ldg", 0, 8, 4, 0) in c
    assert not any(v == "tma" and ty == 16 for v, _, ty, _, _ in c)  # FP32 16-row stages do not fit
    assert all(126 // seg >= 4 for _, _, _, seg, _ in c)
    assert ("tma", 1, 16, 2, 0) in tune.candidates(126, "bf16")
    for cand in c:
        assert tune.parse(tune.name(cand)) == cand
    assert tune.parse("ldg:0:8:4") == ("ldg", 0, 8, 4, 0)


def test_tma_even_splits_and_z_segments():
    """The TMA kernel's candidates include the even row splits whose items fill
    whole waves of its resident CTAs (38 tiles of 3-4 rows x 4 segments = 608
    CTAs, four per SM at 128^3), and the z-segment list the 16-bit step tunes to."""
    c = tune.candidates(126, "f32", nx=128, ny=128, n_sm=152)
    assert ("tma", 1, 4, 4, 38) in c
    for v, ns, ty, seg, nty in c:
        if v == "tma" and nty:
            assert ns == 1 and -(-128 // nty) in (ty - 1, ty)
            assert any((4 * nty * seg) % (152 * k) == 0 for k in tune.TMA_CTAS_PER_SM[ty])
    b = tune.candidates(126, "bf16", nx=256, ny=256, n_sm=152)
    assert ("tma", 1, 8, 7, 0) in b
    assert set(tune.SEGMENTS) >= {1, 2, 3, 4, 6, 7, 8, 12, 16}


def test_batch_candidates_cover_both_kernels():
    variants = {v for v, _, _ in tune.BATCH_CANDIDATES}
    assert variants == {"tma", "ldg"}
    assert all(ty in (4, 8) for v, ty, _ in tune.BATCH_CANDIDATES if v == "tma")  # the TMA batch kernel's tiles
