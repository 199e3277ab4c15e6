"""The pair pass sorts the (key, index) words of swarms of at most 8 with a
fixed network of compare-exchanges (csrc/qs_device.cuh, sort8). By the 0-1
principle (Knuth, TAOCP vol. 3, 5.3.4) a comparator network sorts every input
iff it sorts every sequence of zeros and ones; this test reads the network
from the source and checks all 256 of them, so an edit that drops or swaps a
comparator fails on the CPU before any GPU run."""
import itertools
import pathlib
import re

SRC = pathlib.Path(__file__).resolve().parents[1] / "paper_2306_09537_gb300" / "csrc" / "qs_device.cuh"


def network():
    text = SRC.read_text()
    body = text[text.index("void sort8(uint64_t k[8])"):]
    body = body[:body.index("\n}\n")]
    return [(int(a), int(b)) for a, b in re.findall(r"cmp_swap\(k\[(\d)\], k\[(\d)\]\)", body)]


def apply(net, seq):
    a = list(seq)
    for i, j in net:
        if a[i] > a[j]:
            a[i], a[j] = a[j], a[i]
    return a


def test_network_has_nineteen_comparators_on_eight_wires():
    net = network()
    assert len(net) == 19
    assert all(0 <= i < j < 8 for i, j in net)


def test_network_sorts_every_zero_one_input():
    net = network()
    for bits in itertools.product((0, 1), repeat=8):
        assert apply(net, bits) == sorted(bits), bits


def test_a_dropped_comparator_is_caught():
    """The check itself rejects a broken network: without any one of its
    comparators the network leaves some 0-1 input unsorted."""
    net = network()
    for drop in range(len(net)):
        broken = net[:drop] + net[drop + 1:]
        assert any(apply(broken, bits) != sorted(bits) for bits in itertools.product((0, 1), repeat=8)), drop
