"""Host placement of the benchmark's end-to-end buffers: the NUMA node of
the GPU's PCI function and its CPU list are read from sysfs (a fake tree
here), the calling thread runs on those CPUs while the pinned buffers are
allocated, and its affinity is restored afterwards; unknown nodes change
nothing."""
import os
import sys
import types

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)
import bench  # noqa: E402


def _fake_sysfs(tmp_path, bus, node, cpulist):
    dev = tmp_path / "bus" / "pci" / "devices" / bus
    dev.mkdir(parents=True)
    (dev / "numa_node").write_text(f"{node}\n")
    if node >= 0:
        nd = tmp_path / "devices" / "system" / "node" / f"node{node}"
        nd.mkdir(parents=True)
        (nd / "cpulist").write_text(cpulist + "\n")
    return str(tmp_path)


def test_parse_cpulist():
    assert bench.parse_cpulist("0-3,8,10-11\n") == {0, 1, 2, 3, 8, 10, 11}
    assert bench.parse_cpulist("5") == {5}
    assert bench.parse_cpulist("") == set()


def test_host_node_from_pci_function(tmp_path, monkeypatch):
    import torch
    props = types.SimpleNamespace(pci_domain_id=0x9, pci_bus_id=0x1b, pci_device_id=0x0)
    monkeypatch.setattr(torch.cuda, "get_device_properties", lambda d: props)
    root = _fake_sysfs(tmp_path, "0009:1b:00.0", 1, "0")
    assert bench.host_node_of(0, sysfs=root) == 1


def test_host_node_unknown(tmp_path, monkeypatch):
    import torch
    props = types.SimpleNamespace(pci_domain_id=0, pci_bus_id=0x3, pci_device_id=0x0)
    monkeypatch.setattr(torch.cuda, "get_device_properties", lambda d: props)
    root = _fake_sysfs(tmp_path, "0000:03:00.0", -1, "")
    assert bench.host_node_of(0, sysfs=root) is None          # sysfs says "no node"
    assert bench.host_node_of(0, sysfs=str(tmp_path / "missing")) is None


@pytest.mark.skipif(not hasattr(os, "sched_setaffinity"), reason="no affinity control")
def test_affinity_set_and_restored(tmp_path):
    before = os.sched_getaffinity(0)
    one = min(before)
    nd = tmp_path / "devices" / "system" / "node" / "node3"
    nd.mkdir(parents=True)
    (nd / "cpulist").write_text(f"{one}\n")
    with bench.cpus_of_node(3, sysfs=str(tmp_path)):
        assert os.sched_getaffinity(0) == {one}
    assert os.sched_getaffinity(0) == before
    # CPUs of the node that the process may not use are left out; none usable -> unchanged
    (nd / "cpulist").write_text(f"{max(before) + 1000}\n")
    with bench.cpus_of_node(3, sysfs=str(tmp_path)):
        assert os.sched_getaffinity(0) == before
    with bench.cpus_of_node(None, sysfs=str(tmp_path)):
        assert os.sched_getaffinity(0) == before
    with bench.cpus_of_node(7, sysfs=str(tmp_path)):      # no such node
        assert os.sched_getaffinity(0) == before


def test_host_copy_rates_never_fail_the_bench():
    """The host-link report is a side field: where it cannot be measured (here:
    no GPU) it reports None instead of raising."""
    import torch
    if torch.cuda.is_available():
        pytest.skip("measures on a GPU")
    t = {"x": torch.zeros(4)}
    bufs = {"x": types.SimpleNamespace(send=torch.zeros(4), recv=torch.zeros(4))}
    out = bench.host_copy_rates(t, t, bufs, ["x"], None, "cpu")
    assert out == {"h2d_gbs": None, "d2h_gbs": None, "both_directions_gbs": None}
