"""bench.py --write-counters: per-launch ncu counters of the reported kernel classes from a CSV.

tree, level_big and level_small are one kernel each (one value per launch, averaged); walk is the
predict walk kernel alone; predict is every launch from the query coding to the walk, summed per
call; kernels of other classes (the presort's radix sort, for instance) count for nothing even
when they share a name with a kernel inside the predict call.
"""
import csv
import json

import bench

HDR = ["ID", "Process ID", "Process Name", "Host Name", "Kernel Name", "Context", "Stream", "Block Size",
       "Grid Size", "Device", "CC", "Section Name", "Metric Name", "Metric Unit", "Metric Value"]


def rows_for(lid, name, read, write, unit="byte", inst=None, wf=None):
    base = [str(lid), "1", "python3", "h", name, "1", "7", "(256, 1, 1)", "(1, 1, 1)", "0", "10.3", "Command line"]
    out = [base + ["dram__bytes_read.sum", unit, f"{read:,}"], base + ["dram__bytes_write.sum", unit, f"{write:,}"]]
    if inst is not None:
        out.append(base + ["smsp__inst_executed.sum", "inst", f"{inst:,}"])
    if wf is not None:
        out.append(base + ["l1tex__data_pipe_lsu_wavefronts_mem_shared.sum", "", f"{wf:,}"])
    return out


def write_csv(path, launches):
    with open(path, "w", newline="") as fh:
        fh.write("==PROF== Connected to process\n")
        w = csv.writer(fh)
        w.writerow(HDR)
        for i, launch in enumerate(launches):
            for row in rows_for(i, *launch):
                w.writerow(row)


def test_classes_and_sums(tmp_path):
    launches = [
        ("void aiwcrf::sort_hist_kernel(const unsigned int *, long, long, int, int, unsigned int *)", 1000, 1000),
        ("aiwcrf::tree_grow_kernel(aiwcrf::TreeArgs)", 70, 30, "byte", 9_000_000),
        ("void aiwcrf::level_big_kernel<unsigned char>(aiwcrf::LevelArgs, int)", 100, 20),
        ("void aiwcrf::level_small_kernel<unsigned char>(aiwcrf::LevelArgs)", 50, 10),
        ("void aiwcrf::level_big_kernel<unsigned char>(aiwcrf::LevelArgs, int)", 300, 60),
        ("void aiwcrf::level_small_kernel<unsigned char>(aiwcrf::LevelArgs)", 150, 30),
        ("void aiwcrf::finalize_kernel(aiwcrf::FinalArgs)", 5, 5),
        ("void aiwcrf::code_queries_kernel<unsigned char>(const float *, long, int, const float *, long, "
         "const unsigned int *, T1 *, int)", 128_000, 36_000),
        ("aiwcrf::query_key_kernel(const unsigned char *, int, long, int4, unsigned int *, unsigned int *)", 36, 8),
        ("void aiwcrf::sort_hist_kernel(const unsigned int *, long, long, int, int, unsigned int *)", 8, 1),
        ("void aiwcrf::predict4_kernel<2, 0, 1>(const unsigned int *, const long *)", 40, 8, "byte", 5_000, 700),
        ("void aiwcrf::serve_select_kernel<1>(aiwcrf::ServeForest)", 7, 7),
    ]
    path = tmp_path / "t.csv"
    write_csv(path, launches)
    out = tmp_path / "counters.json"
    d = bench.write_counters(str(path), "ncu ...", str(out))
    saved = json.load(open(out))
    assert set(saved) == set(d) and all(saved[c]["commands"] == ["ncu ..."] for c in d)
    assert d["level_big"]["launches"] == 2 and d["level_big"]["dram_bytes"] == (120 + 360) / 2
    assert d["level_small"]["launches"] == 2 and d["level_small"]["dram_bytes"] == (60 + 180) / 2
    assert d["tree"]["dram_bytes"] == 100 and d["tree"]["inst"] == 9_000_000
    assert d["walk"]["inst"] == 5_000 and d["walk"]["smem_wavefronts"] == 700 and d["walk"]["dram_bytes"] == 48
    # predict: coding + key + the key sort's kernel + the walk; not the presort's sort kernel
    assert d["predict"]["launches"] == 1
    assert d["predict"]["dram_bytes"] == 164_000 + 44 + 9 + 48
    assert set(d) == {"level_big", "level_small", "tree", "walk", "predict"}
    assert all(v["source_sha"] == bench.source_sha(c) for c, v in d.items())


def test_units_scale_and_merge(tmp_path):
    path = tmp_path / "t.csv"
    write_csv(path, [("void aiwcrf::level_small_kernel<unsigned short>(aiwcrf::LevelArgs)", 1.5, 0.5, "Mbyte")])
    o = tmp_path / "o.json"
    o.write_text(json.dumps({"walk": {"inst": 3, "source_sha": "x"},
                             "level_small": {"inst": 7, "source_sha": bench.source_sha("level_small"), "command": "a"}}))
    d = bench.write_counters(str(path), "b", str(o))
    assert d["level_small"]["dram_bytes"] == 2_000_000
    saved = json.load(open(o))
    assert set(saved) == {"walk", "level_small"}                        # earlier captures are kept
    assert saved["level_small"]["inst"] == 7 and saved["level_small"]["commands"] == ["a", "b"]   # merged


def test_scaled_capture_keeps_instruction_counts_only(tmp_path):
    path = tmp_path / "t.csv"
    write_csv(path, [("aiwcrf::tree_grow_kernel(aiwcrf::TreeArgs)", 70, 30, "byte", 1000, 40)])
    d = bench.write_counters(str(path), "c", str(tmp_path / "o.json"), scale={"tree": 8.0})
    assert d["tree"]["inst"] == 8000 and d["tree"]["smem_wavefronts"] == 320 and "dram_bytes" not in d["tree"]


def test_counters_reported_only_for_the_captured_sources(tmp_path):
    p = tmp_path / "counters.json"
    p.write_text(json.dumps({"predict": {"dram_bytes": 1.5e8, "source_sha": "abc", "launches": 1}}))
    assert bench.ncu_traffic("predict", "abc", str(p)) == 1.5e8
    assert bench.ncu_traffic("predict", "abd", str(p)) is None          # kernels changed since
    assert bench.ncu_traffic("level_small", "abc", str(p)) is None      # not captured
    assert bench.ncu_counter("predict", "inst", "abc", str(p)) is None
    assert bench.ncu_traffic("predict", "abc", str(tmp_path / "missing.json")) is None
