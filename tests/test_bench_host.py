"""Host logic of bench.py that decides whether a stored ncu traffic figure still
applies: the hash of the step kernels' code ignores comments and blank lines but
not the code itself."""
import hashlib

import bench


def _hash(text: str) -> str:
    return hashlib.sha256(bench.code_only(text).encode()).hexdigest()


def test_code_only_drops_comments_and_blank_lines():
    src = "int a = 1;  // one\n\n/* block\n   comment */\nint b = a * 2; /* inline */\n"
    assert bench.code_only(src) == "int a = 1;\nint b = a * 2;"


def test_comment_edits_keep_the_hash_and_code_edits_change_it():
    with open(bench.os.path.join(bench.ROOT, bench.KERNEL_SOURCES[0]), encoding="utf-8") as fh:
        src = fh.read()
    commented = src.replace("\n", "\n// an added remark\n", 3) + "\n/* trailing note */\n\n"
    assert _hash(commented) == _hash(src)
    changed = src.replace("kTileX = 32", "kTileX = 64", 1)
    assert changed != src and _hash(changed) != _hash(src)


def test_traffic_table_matches_the_current_kernel_code():
    """The traffic figure reported next to the roofline is keyed by the code hash;
    the table holds one for the kernel the benchmark times in its layout."""
    keys = {k for k in bench.NCU_TRAFFIC if k[0] == "k_step_tma_dyn<f2>" and k[1] == "rows"}
    assert (("k_step_tma_dyn<f2>", "rows", bench.kernel_source_hash()) in keys)


def test_d3q19_traffic_table_matches_the_current_kernel_code():
    """The D3Q19 step's stored ncu traffic is keyed by the hash of csrc/lbm3d.cu."""
    sha = bench.kernel_source_hash(bench.KERNEL_SOURCES_D3Q19)
    assert ("k_d3_step<float, true>", sha) in bench.NCU_TRAFFIC_D3Q19
    assert sha != bench.kernel_source_hash()
