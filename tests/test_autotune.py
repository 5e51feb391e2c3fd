"""The autotuner's bookkeeping (no GPU): every candidate shape is built and
timed, the fastest is recorded per workload, and the build takes the
defines of the workload named by ``use``."""
import json


def test_tuner_records_the_fastest_shape(tmp_path):
    from paper_2410_23802_gb300 import autotune as A, build as B
    path = str(tmp_path / "tuned.json")
    built = []
    times = {"tune_y4": 1.30, "tune_y2": 1.25, "tune_y8": 1.40, "tune_y4_b6": 1.35, "tune_y4_p1": 1.31,
             "tune_y8_p1": 1.41}

    def fake_build(defines, out):
        built.append((tuple(defines), out))

    def fake_timer(lib, workload, steps):
        tag = lib.rsplit("/", 1)[-1][:-3]
        return {"ms_per_step": times[tag], "cells": 1000}

    rec = A.tune("channels", steps=7, path=path, build=fake_build, timer=fake_timer)
    assert len(built) == len(A.CANDIDATES) == len({b[1] for b in built})
    assert ("VLB_TILE_Y=4", "VLB_BATCH_PERSISTENT=1") in [b[0] for b in built]
    y2 = ["VLB_TILE_Y=2"]
    assert rec["channels"]["defines"] == y2 and rec["use"] == "channels"
    assert B.tuned_defines(path) == y2
    # a second workload recorded without taking over the build's choice
    times["tune_y8"] = 0.5
    built.clear()
    rec = A.tune("cavity", steps=7, path=path, use=False, build=fake_build, timer=fake_timer)
    assert len(built) == 4  # the batched-step form is not timed on a single case
    assert rec["cavity"]["defines"] == ["VLB_TILE_Y=8"] and rec["use"] == "channels"
    assert B.tuned_defines(path) == y2
    r = json.load(open(path))["cavity"]["results"]
    assert abs(r[2]["mlups"] - 1000 / 0.5e-3 / 1e6) < 1e-12


def test_candidates_are_valid_builds():
    from paper_2410_23802_gb300 import autotune as A
    tags = set()
    for ty, mb, pers in A.CANDIDATES:
        assert ty in (1, 2, 4, 8) and 32 * ty <= 1024
        assert mb is None or 1 <= mb <= 1024 // (32 * ty)
        assert pers in (None, 0, 1)
        tags.add(A.candidate_tag(A.candidate_defines(ty, mb, pers)))
    assert len(tags) == len(A.CANDIDATES)


def test_missing_or_broken_tuned_file_means_no_defines(tmp_path):
    from paper_2410_23802_gb300 import build as B
    assert B.tuned_defines(str(tmp_path / "none.json")) == []
    bad = tmp_path / "bad.json"
    bad.write_text("{\"use\": \"cavity\"}")
    assert B.tuned_defines(str(bad)) == []
