"""Host helpers of bench.py on the CPU: the kernel-source hash that keys the
recorded ncu counters ignores comments and blank lines but not code."""
import bench


def test_code_only_drops_comments_and_keeps_code():
    src = 'int a = 1;  // one\n/* block\n comment */\n\nconst char* s = "x // y"; // z\n'
    assert bench._code_only(src) == 'int a = 1;\nconst char* s = "x // y";'
    assert bench._code_only("int a = 1; // one") == bench._code_only("int a = 1; // two")
    assert bench._code_only("int a = 1;") != bench._code_only("int a = 2;")


def test_recorded_counters_are_keyed_by_the_hash():
    sha = bench.kernel_source_sha()
    assert len(sha) == 16 and all(c in "0123456789abcdef" for c in sha)


def test_recorded_counters_match_the_current_kernels():
    """profiles/kernel_counters.txt holds ncu counters of the dominant kernel
    for the kernel sources as they are (else the bench would report no
    traffic): a kernel change must come with a new capture."""
    c = bench.kernel_counters("k_p2g_g2p_bwd")
    assert c is not None, bench.kernel_source_sha()
    assert c["dram_bytes"] > 0 and c["warp_insts"] > 0
