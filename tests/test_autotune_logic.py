"""Host logic of the autotuner: size classes, the moduli choice from a calibration table, and
the residue-GEMM configuration choice from timings (no GPU)."""
from paper_2606_29129_gb300 import autotune
from paper_2606_29129_gb300 import ozaki2 as oz


class FakeHandle:
    def __init__(self):
        self.options = {}

    def set_option(self, option, value):
        self.options[option] = value


def test_size_classes():
    assert autotune.size_class(1) == 0
    assert autotune.size_class(64) == 0
    assert autotune.size_class(65) == 1
    assert autotune.size_class(16384) == len(autotune.CLASS_EDGES) - 1
    assert autotune.size_class(10 ** 6) == len(autotune.CLASS_EDGES) - 1


def test_choose_n_equal_accuracy_and_target():
    table = {3: {"k": 512, "cublas": 1e-11, "N": {13: 5e-10, 14: 2e-11, 15: 9e-12, 16: 1e-14}}}
    assert autotune.choose_n(table, 500) == 15            # smallest N not worse than cuBLAS
    assert autotune.choose_n(table, 500, target=1e-13) == 16
    assert autotune.choose_n(table, 500, target=1e-20) == 16   # none meets it: the largest
    assert autotune.choose_n(table, 5000) == 16           # class not calibrated: the default


def test_best_config_and_apply():
    ms = {(oz.GEMM_SINGLE, 960): 3.0, (oz.GEMM_PAIR, 960): 2.5, (oz.GEMM_SINGLE, 640): 2.5}
    assert autotune.best_config(ms) == (oz.GEMM_PAIR, 960)   # fastest, first listed on a tie
    table = {autotune.size_class(4096): {"size": 4096, "ms": ms, "best": (oz.GEMM_PAIR, 960)}}
    h = FakeHandle()
    assert autotune.apply_tiles(h, table, 4096)
    assert h.options == {oz.OPT_GEMM_VARIANT: oz.GEMM_PAIR, oz.OPT_CHUNK_K: 960,
                         oz.OPT_GROUP_M: 0}
    table3 = {autotune.size_class(4096): {"size": 4096, "ms": {}, "best": (oz.GEMM_SINGLE, 640, 32)}}
    h3 = FakeHandle()
    assert autotune.apply_tiles(h3, table3, 4096) and h3.options[oz.OPT_GROUP_M] == 32
    assert autotune.tiles_to_json(table3)[str(autotune.size_class(4096))]["best"]["group_m"] == 32
    h2 = FakeHandle()
    assert not autotune.apply_tiles(h2, table, 64) and h2.options == {}
    js = autotune.tiles_to_json(table)
    assert js[str(autotune.size_class(4096))]["best"] == {"variant": oz.GEMM_PAIR, "chunk_k": 960}


class FakeGroupedHandle:
    def __init__(self):
        self.rules = []

    def set_grouped_tiles(self, rules):
        self.rules = list(rules)


def test_tune_grouped_tiles_coordinate_descent(monkeypatch):
    """The per-class tuner keeps, class by class, the tile width and chunk that time fastest;
    with a cost that is a sum of independent per-class costs it reaches the optimum."""
    best_width = {64: 64, 128: 64, 256: 128, 512: 256, 1 << 30: 256}
    best_chunk = {64: 0, 128: 0, 256: 640, 512: 448, 1 << 30: 960}
    h = FakeGroupedHandle()

    def cost(rules):
        if not rules:                     # the automatic configuration
            return 100.0
        t = 0.0
        for n_max, _, tn, ck in rules:
            t += 1.0 + (tn != best_width[n_max]) * 2.0 + (ck != best_chunk[n_max]) * 0.5
        return t

    monkeypatch.setattr(autotune, "_time_ms", lambda call, reps: cost(h.rules))
    res = autotune.tune_grouped_tiles(lambda: None, h)
    got = {r[0]: (r[2], r[3]) for r in res["rules"]}
    assert got == {e: (best_width[e], best_chunk[e] if best_chunk[e] else 0)
                   for e in autotune.GROUPED_N_EDGES}
    assert h.rules == res["rules"] and res["best_ms"] == 5.0 and res["auto_ms"] == 100.0


def test_tune_grouped_tiles_keeps_automatic_when_not_beaten(monkeypatch):
    h = FakeGroupedHandle()
    monkeypatch.setattr(autotune, "_time_ms", lambda call, reps: 1.0 if not h.rules else 2.0)
    res = autotune.tune_grouped_tiles(lambda: None, h)
    assert res["rules"] == [] and h.rules == [] and res["best_ms"] == 1.0


def test_choose_n_margin_and_table_file(tmp_path):
    import json

    table = {3: {"k": 512, "cublas": 1e-11, "N": {13: 5e-10, 14: 2e-11, 15: 9e-12, 16: 1e-14}}}
    assert autotune.choose_n(table, 500, margin=8.0) == 16     # 9e-12 > 1e-11 / 8
    assert autotune.choose_n(table, 500, target=1e-13, margin=8.0) == 16
    path = tmp_path / "cal.json"
    path.write_text(json.dumps({"table": autotune.table_to_json(table)}))
    assert autotune.load_calibration(str(path)) == table
    assert autotune.load_calibration(str(tmp_path / "missing.json")) is None
