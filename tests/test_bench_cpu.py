"""Host-side logic of bench.py that a GPU run depends on: the residue-pass
count of the large-prime block line, and the DRAM traffic records, which
must turn to null once a kernel's sources change."""
import hashlib
import json
import os

import pytest

import bench


def _primes_desc(limit, count):
    out, c = [], limit
    while len(out) < count:
        if c > 1 and all(c % d for d in range(2, int(c ** 0.5) + 1)):
            out.append(c)
        c -= 1
    return out


@pytest.mark.parametrize("p,k", [(65521, 16384), (65791, 16384), (65797, 16384), (2147483647, 16384),
                                 (4294967291, 16384), (4294967291, 1), (1000003, 100000)])
@pytest.mark.parametrize("direct_max", [65791, 65536])
def test_rns_passes_is_the_minimal_cover(p, k, direct_max):
    """Residue moduli are the largest primes <= 65536; the direct range is
    p <= 65791 for uint32 A and p <= 65536 for a prepared A."""
    L = bench.rns_passes(p, k, direct_max)
    if p <= direct_max:
        assert L == 1
        return
    primes = _primes_desc(65536, 8)
    bound = k * (p - 1) ** 2
    prod = 1
    for q in primes[:L]:
        prod *= q
    assert prod > bound                      # the residues fix every entry sum
    assert prod // primes[L - 1] <= bound    # one modulus fewer would not


def test_traffic_records_follow_their_sources(tmp_path, monkeypatch):
    src = tmp_path / "k.cu"
    src.write_text("kernel v1\n")
    (tmp_path / "profiles").mkdir()
    rec = {"k_test": {"sources": ["k.cu"], "sha256": hashlib.sha256(b"kernel v1\n").hexdigest(),
                      "dram_bytes_per_algorithmic_byte": 1.25}}
    (tmp_path / "profiles" / "traffic.json").write_text(json.dumps(rec))
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    assert bench.traffic_for("k_test", 1000.0) == pytest.approx(1250.0)
    assert bench.traffic_for("k_other", 1000.0) is None
    # comment lines and lines only a device-checks build compiles leave the record valid
    src.write_text("kernel v1\n\n    GFP_DCHECK(w, c, 1u);\n#ifdef GFP_DEVICE_CHECKS\nx\n#endif\n"
                   "    // a comment\n")
    assert bench.traffic_for("k_test", 1000.0) == pytest.approx(1250.0)
    src.write_text("kernel v2\n")            # the kernel changed since the capture
    assert bench.traffic_for("k_test", 1000.0) is None


def test_committed_traffic_records_name_existing_sources():
    path = os.path.join(bench.ROOT, "profiles", "traffic.json")
    recs = json.load(open(path))
    assert recs
    for name, rec in recs.items():
        assert name.startswith("k_")
        assert 0.5 < rec["dram_bytes_per_algorithmic_byte"] < 2.0
        for f in rec["sources"]:
            assert os.path.exists(os.path.join(bench.ROOT, f)), (name, f)
