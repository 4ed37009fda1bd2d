"""The committed ncu summaries carry the figures the benchmark reads for its
roofline objects, and each names the command that produced it."""
import os

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_benchmark_figures_present():
    import bench
    for name, key in (("k_walk_generation_200x1e6.md", "traffic_bytes_per_child"),
                      ("k_eval_items_full_eval_100x1e6.md", "traffic_bytes_per_node"),
                      ("k_copy_children_fitness_first_200x1e6.md", "traffic_per_algorithmic_byte"),
                      ("crossover_dram_traffic_100x1e6.md", "traffic_per_algorithmic_byte")):
        v = bench.profile_figure(name, key)
        assert v is not None and v > 0, (name, key)


def test_every_summary_names_its_command():
    d = os.path.join(ROOT, "profiles")
    names = sorted(os.listdir(d))
    assert names
    for n in names:
        assert n.endswith((".md", ".txt")), n
        text = open(os.path.join(d, n)).read()
        assert "ncu " in text and "--clock-control none" in text, n
        assert "python bench.py" in text, n
