"""The per-region FP64 instruction counts behind the benchmark's roofline
(bench.py RULE_FP64_INST_D8) were taken by ncu on one version of the FP64
rule kernel.  They stay valid only while that kernel's sources are
unchanged: this check fails as soon as they change, until the counts are
taken again (bench.py --probe-rule under ncu, as profiles/rule_fp64_d8.md
gives the command) and the fingerprint is updated with them."""
import bench


def test_rule_counts_belong_to_the_current_kernel_sources():
    assert bench.rule_source_fingerprint() == bench.RULE_COUNTS_SHA16, (
        "the FP64 rule kernel changed since its instruction counts were taken")


def test_counts_cover_the_benchmark_families():
    from paper_2511_01573_gb300 import genz_inputs as G
    for fam in G.GENZ_D8_FAMILIES:
        assert bench.RULE_FP64_INST_D8[fam] > 401 and bench.RULE_FP64_FLOPS_D8[fam] > 401


def test_mixed_counts_belong_to_the_current_kernel_sources():
    assert (bench.rule_source_fingerprint(bench.MIXED_COUNTS_SOURCES) ==
            bench.MIXED_COUNTS_SHA16), (
        "the mixed rule kernel changed since its FP32 operation counts were taken")
