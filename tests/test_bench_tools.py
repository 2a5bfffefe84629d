"""Host-side helpers of bench.py: kernel-name grouping and the per-kernel
summary of an ncu launch list (no GPU needed)."""
import bench


def test_kernel_names_match_whole_identifiers():
    assert bench.short("srn::<unnamed>::digit_scan_kernel(unsigned int *, int, unsigned int *)") == \
        "srn::digit_scan_kernel"
    assert bench.short("srn::<unnamed>::scan_kernel(unsigned int *, int, int, const unsigned int *)") == \
        "srn::scan_kernel"
    assert bench.short("void srn::mma::render_mma_kernel<32, 14, 16, 1, 0, 0, 0>(NetDev, BatchDev)") == \
        "srn::render_mma_kernel"
    # unknown kernels of ours keep their template arguments; library kernels lose them
    assert bench.short("void srn::<unnamed>::fit_mma_kernel<12, 8, 0>(NetDev)") == \
        "srn::<unnamed>::fit_mma_kernel<12, 8, 0>"
    assert bench.short("void at::native::vectorized_elementwise_kernel<4, float>(int)") == \
        "at::native::vectorized_elementwise_kernel"


def test_summarize_launches(tmp_path, capsys):
    rows = [("1", "srn::<unnamed>::digit_scan_kernel(unsigned int *)", "usecond", "2"),
            ("2", "srn::<unnamed>::digit_scan_kernel(unsigned int *)", "usecond", "2"),
            ("3", "void srn::mma::render_mma_kernel<32>(NetDev)", "msecond", "1.5"),
            ("4", "srn::<unnamed>::scan_kernel(unsigned int *)", "nsecond", "1,000")]
    lines = ['==PROF== Connected to process 1',
             '"ID","Kernel Name","Metric Name","Metric Unit","Metric Value"']
    lines += [f'"{i}","{k}","gpu__time_duration.sum","{u}","{v}"' for i, k, u, v in rows]
    lines.append('"5","other","dram__bytes_read.sum","byte","9"')
    p = tmp_path / "launches.csv"
    p.write_text("\n".join(lines) + "\n")
    bench.summarize_launches(str(p))
    out = capsys.readouterr().out.splitlines()
    table = {ln.split()[0]: ln.split()[1:] for ln in out[1:]}
    assert table["srn::render_mma_kernel"][:2] == ["1", "1.500"]
    assert table["srn::digit_scan_kernel"][:2] == ["2", "0.004"]
    assert table["srn::scan_kernel"][:2] == ["1", "0.001"]
    assert table["all"] == ["4", "1.505"]
