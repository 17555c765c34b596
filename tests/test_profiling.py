"""The ncu CSV summaries of paper_1611_00463_gb300.profiling on a small
hand-written launch list (no GPU): per-kernel totals, the whole-sort cut and
the last sort's launches in order."""
from paper_1611_00463_gb300 import profiling

CSV = '''==PROF== Connected to process 1
"ID","Process ID","Process Name","Host Name","Kernel Name","Context","Stream","Block Size","Grid Size","Device","CC","Section Name","Metric Name","Metric Unit","Metric Value"
"0","1","python","h","void pgs::k_block_sort<unsigned int, 1>(const T1 *)","1","7","(256, 1, 1)","(4, 1, 1)","0","10.3","Command line profiler metrics","gpu__time_duration.sum","us","20.00"
"1","1","python","h","void pgs::k_merge_tile<unsigned int, 1, 128, 17>(const T1 *)","1","7","(128, 1, 1)","(8, 1, 1)","0","10.3","Command line profiler metrics","gpu__time_duration.sum","ns","8000"
"2","1","python","h","pgs::k_stats(pgs::Geo)","1","7","(256, 1, 1)","(1, 1, 1)","0","10.3","Command line profiler metrics","gpu__time_duration.sum","us","4.00"
"3","1","python","h","void pgs::k_block_sort<unsigned int, 1>(const T1 *)","1","7","(256, 1, 1)","(4, 1, 1)","0","10.3","Command line profiler metrics","gpu__time_duration.sum","us","22.00"
"4","1","python","h","pgs::k_stats(pgs::Geo)","1","7","(256, 1, 1)","(1, 1, 1)","0","10.3","Command line profiler metrics","gpu__time_duration.sum","us","3.00"
"5","1","python","h","void pgs::k_block_sort<unsigned int, 1>(const T1 *)","1","7","(256, 1, 1)","(4, 1, 1)","0","10.3","Command line profiler metrics","gpu__time_duration.sum","us","99.00"
'''


def _write(tmp_path):
    p = tmp_path / "launches.csv"
    p.write_text(CSV)
    return str(p)


def test_whole_sorts_totals(tmp_path):
    out = profiling.launches(_write(tmp_path), whole_sorts=True).splitlines()
    rows = {ln.split()[0]: ln.split() for ln in out[1:]}
    assert rows["k_block_sort<u32,1>"][1:3] == ["2", "42.0"]          # the cut-off third sort is dropped
    assert rows["k_merge_tile<u32,1,128,17>"][1:3] == ["1", "8.0"]   # ns converted to us
    assert rows["total"][1:3] == ["5", "57.0"]


def test_last_sort_in_order(tmp_path):
    out = profiling.last_sort(_write(tmp_path)).splitlines()
    assert [ln.split()[0] for ln in out] == ["k_block_sort<u32,1>", "k_stats", "total"]
    assert out[0].split()[1] == "22.00" and "grid (4, 1, 1)" in out[0]
    assert out[-1].split()[1] == "25.00" and out[-1].endswith("2 launches")
