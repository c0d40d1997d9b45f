"""The synthetic inputs follow their stated recipe.

Every workload is drawn from splitmix64 (Steele, Lea, Flood, "Fast splittable
pseudorandom number generators", OOPSLA 2014).  These checks fix the
generator to the published outputs of that algorithm, and each workload
builder to the distribution and the structure it claims:
  - tiny pairs: 1,000 blocking int32 sends of U[1, 4096] elements with tags
    U[0, 7], received by blocking receives in a random order that keeps each
    tag's order;
  - ring exchange (§6, Listing 4's axpy between the exchanges): sizes
    log-uniform over 4 KB - 64 MB, the four layout pairs equally likely, the
    vector type MPI_Type_vector(nb, 64, 128) of fp32;
  - batching: sizes log-uniform 8 B - 64 KB, dtypes uniform over
    {uint8, int32, fp32}, tags uniform 0-31, 5 % ANY_TAG and 2 % ANY_SOURCE
    receives, exact receives of a domain posted before its wildcards;
  - 3-D halo: the x, y and z faces of a sub^3 fp32 block as
    vector(sub*sub, 1, sub), vector(sub, sub, sub*sub) and a contiguous plane,
    sent across a periodic 2x2x2 decomposition;
  - allreduce inputs: int64 round(N(0,1) * 2^40), fp32 N(0,1), int32 over the
    full range;
  - serving: Zipf(1.2) power-of-two sizes, 30 % allreduce calls, a tag that
    counts each (source, destination) pair's messages.
Statistical checks use fixed seeds and bounds of five standard deviations
(or the 0.1 % Kolmogorov-Smirnov quantile), so they either always pass or
always fail.  CPU only."""
import math

import numpy as np
import pytest

from traffic import gen
from traffic.program import (ALLREDUCE, ANY_SOURCE, ANY_TAG, AXPY, IRECV, ISEND, MODE_FIXED,
                             MODE_TREE, RECV, SEND, T_BYTE, T_FLOAT, T_INT32, T_INT64, WAITALL,
                             type_size)
from traffic.rng import Rng


def _raw_stream(state):
    """A splitmix64 generator whose state is `state` (no key derivation)."""
    r = Rng(0)
    r.stream = np.uint64(state)
    r.counter = 0
    return r


def _within(count, n, p, sigmas=5.0):
    """count ~ Binomial(n, p) within `sigmas` standard deviations."""
    sd = math.sqrt(n * p * (1 - p))
    return abs(count - n * p) <= sigmas * sd + 1


def _log2_bins_uniform(sizes, lo_log2, hi_log2):
    """Sizes drawn log-uniformly over [2^lo, 2^hi] fall in each octave
    [2^k, 2^(k+1)) with probability 1 / (hi - lo).  Rounding a size down to a
    multiple of 4 or 256 keeps it in its octave (every 2^k >= 256 is such a
    multiple; below 256 only 4-byte rounding applies and 2^k >= 8)."""
    sizes = np.asarray(sizes, np.int64)
    assert sizes.min() >= (1 << lo_log2) and sizes.max() <= (1 << hi_log2)
    k = np.floor(np.log2(sizes)).astype(np.int64)
    k = np.minimum(k, hi_log2 - 1)          # the top value 2^hi belongs to the last octave
    nb = hi_log2 - lo_log2
    counts = np.bincount(k - lo_log2, minlength=nb)
    bad = [(lo_log2 + j, int(c)) for j, c in enumerate(counts) if not _within(c, len(sizes), 1.0 / nb)]
    assert not bad, f"octaves off a log-uniform draw (octave, count of {len(sizes)}): {bad}"


# ---------------------------------------------------------------------------
# the generator
# ---------------------------------------------------------------------------
def test_splitmix64_matches_published_outputs():
    """The reference splitmix64 outputs for states 0 and 1234567."""
    assert [int(x) for x in _raw_stream(0).u64(4)] == [
        0xE220A8397B1DCDAF, 0x6E789E6AA1B965F4, 0x06C45D188009454F, 0xF88BB8A8724C81EC]
    assert [int(x) for x in _raw_stream(1234567).u64(5)] == [
        6457827717110365317, 3203168211198807973, 9817491932198370423,
        4593380528125082431, 16408922859458223821]


def test_generator_is_counter_based():
    """Draw i of a stream does not depend on how the draws before it were split."""
    a = Rng(gen.SEED_BASE, 7, 3).u64(1000)
    r = Rng(gen.SEED_BASE, 7, 3)
    b = np.concatenate([r.u64(1), r.u64(499), r.u64(500)])
    assert np.array_equal(a, b)
    assert not np.array_equal(a, Rng(gen.SEED_BASE, 7, 4).u64(1000))


def test_uniform_integers_and_normal_draws():
    n = 200_000
    u = Rng(gen.SEED_BASE, 1).uniform(n)
    assert u.min() >= 0.0 and u.max() < 1.0
    assert abs(u.mean() - 0.5) < 5 * math.sqrt(1 / 12 / n)
    ints = Rng(gen.SEED_BASE, 2).integers(0, 3, n)
    assert set(np.unique(ints)) == {0, 1, 2, 3}
    assert all(_within(int(c), n, 0.25) for c in np.bincount(ints))
    z = np.sort(Rng(gen.SEED_BASE, 3).normal(n))
    phi = 0.5 * (1.0 + np.frompyfunc(math.erf, 1, 1)(z / math.sqrt(2.0)).astype(np.float64))
    i = np.arange(1, n + 1)
    d = max(np.max(i / n - phi), np.max(phi - (i - 1) / n))
    assert d < 1.95 / math.sqrt(n), f"Box-Muller draws: KS distance {d:.5f} from N(0,1)"


# ---------------------------------------------------------------------------
# tiny pairs
# ---------------------------------------------------------------------------
def test_tiny_pairs_recipe():
    nmsg = 1000
    p = gen.tiny_pairs(nmsg=nmsg)
    s0 = p.ops[p.stream_op_lo[0]: p.stream_op_lo[1]]
    s1 = p.ops[p.stream_op_lo[1]: p.stream_op_lo[2]]
    assert len(s0) == len(s1) == nmsg
    assert np.all(s0["kind"] == SEND) and np.all(s1["kind"] == RECV)
    assert np.all(s0["type"] == T_INT32) and np.all(s0["peer"] == 1) and np.all(s1["peer"] == 0)
    counts, tags, order = p.meta["counts"], p.meta["tags"], p.meta["recv_order"]
    assert counts.min() >= 1 and counts.max() <= 4096
    assert abs(counts.mean() - 2048.5) < 5 * math.sqrt((4096 ** 2 - 1) / 12 / nmsg)
    tc = np.bincount(tags, minlength=8)
    assert len(tc) == 8 and all(_within(int(c), nmsg, 1 / 8) for c in tc)
    assert sorted(order) == list(range(nmsg))
    # each receive names exactly its message, and a tag's messages are received in send order
    assert np.array_equal(s1["count"], counts[order]) and np.array_equal(s1["tag"], tags[order])
    for t in range(8):
        mine = [int(m) for m in order if tags[m] == t]
        assert mine == sorted(mine)
    # the interleaving of the tags is random: most receives are out of send order
    assert np.count_nonzero(np.asarray(order) != np.arange(nmsg)) > nmsg // 2


# ---------------------------------------------------------------------------
# ring exchange
# ---------------------------------------------------------------------------
def test_ring_message_sizes_and_layouts():
    """The full-size ring's draws: 8 ranks x 2 directions x 400 steps."""
    seed = gen.SEED_BASE + 1
    sizes, layouts = [], []
    for step in range(400):
        for r in range(8):
            for d in range(2):
                nbytes, layout = gen._ring_message(seed, step, r, d, 4096, 64 << 20)
                assert nbytes % (4 if layout == 0 else 256) == 0
                sizes.append(nbytes)
                layouts.append(layout)
    _log2_bins_uniform(sizes, 12, 26)
    counts = np.bincount(layouts, minlength=4)
    assert len(counts) == 4 and all(_within(int(c), len(layouts), 0.25) for c in counts)


def test_bench_times_the_ring_recipe():
    bench = pytest.importorskip("bench")
    assert (bench.RANKS, bench.N_AXPY, bench.MIN_BYTES, bench.MAX_BYTES) == (8, 1 << 24, 4096, 64 << 20)
    assert bench.ALPHA == 0.5 and bench.SEED == gen.SEED_BASE + 1


def test_ring_program_structure():
    """Per step and rank: axpy, isend right (tag 0), isend left (tag 1), irecv
    from the left (tag 0), irecv from the right (tag 1), waitall of the four;
    each receive holds exactly the bytes its sender sends; vector layouts are
    fp32 MPI_Type_vector(nb, 64, 128)."""
    R, n, steps = 5, 1000, 6
    p = gen.ring_exchange(nranks=R, n=n, steps=steps, min_bytes=4096, max_bytes=1 << 18)
    assert p.nstreams == R and p.ncomms == 1
    for t in range(5, len(p.types)):
        rec = p.types[t]
        assert (int(rec["kind"]), int(rec["base"]), int(rec["blocklen"]), int(rec["stride"])) == (1, T_FLOAT, 64, 128)
    sent = {}
    for r in range(R):
        ops = p.ops[p.stream_op_lo[r]: p.stream_op_lo[r + 1]]
        assert len(ops) == 6 * steps
        for s in range(steps):
            o = ops[6 * s: 6 * s + 6]
            assert [int(k) for k in o["kind"]] == [AXPY, ISEND, ISEND, IRECV, IRECV, WAITALL]
            assert int(o[0]["count"]) == n and float(o[0]["alpha"]) == 0.5
            assert (int(o[1]["peer"]), int(o[1]["tag"])) == ((r + 1) % R, 0)
            assert (int(o[2]["peer"]), int(o[2]["tag"])) == ((r - 1) % R, 1)
            assert (int(o[3]["peer"]), int(o[3]["tag"])) == ((r - 1) % R, 0)
            assert (int(o[4]["peer"]), int(o[4]["tag"])) == ((r + 1) % R, 1)
            assert int(o[5]["req_n"]) == 4
            for j in (1, 2):
                sent[(s, r, int(o[j]["tag"]))] = type_size(p.types, int(o[j]["type"])) * int(o[j]["count"])
    for r in range(R):
        ops = p.ops[p.stream_op_lo[r]: p.stream_op_lo[r + 1]]
        for s in range(steps):
            for j in (3, 4):
                o = ops[6 * s + j]
                cap = type_size(p.types, int(o["type"])) * int(o["count"])
                assert cap == sent[(s, int(o["peer"]), int(o["tag"]))]
    assert p.meta["payload_bytes"] == sum(sent.values())


# ---------------------------------------------------------------------------
# batching
# ---------------------------------------------------------------------------
def _recvs(p):
    return p.ops[p.ops["kind"] == IRECV]


@pytest.mark.parametrize("laminar", [True, False])
def test_batching_mix(laminar):
    nmsg = 20000
    p = gen.batching(nranks=64, streams_per_rank=4, nmsg=nmsg, max_bytes=1 << 16, laminar=laminar)
    assert p.nstreams == 256 and p.ncomms == 4
    for c in range(4):      # comm c holds every rank's c-th stream
        assert [int(p.stream_rank[g]) for g in p.comm_stream[c]] == list(range(64))
        assert all(int(g) % 4 == c for g in p.comm_stream[c])
    _log2_bins_uniform(p.meta["nbytes"], 3, 16)
    sends = p.ops[p.ops["kind"] == ISEND]
    rv = _recvs(p)
    assert len(sends) == len(rv) == nmsg
    types = np.bincount(sends["type"], minlength=5)
    assert types[T_INT64] == 0 and types[4] == 0
    assert all(_within(int(types[t]), nmsg, 1 / 3) for t in (T_BYTE, T_INT32, T_FLOAT))
    tags = np.bincount(sends["tag"], minlength=32)
    assert len(tags) == 32 and all(_within(int(c), nmsg, 1 / 32) for c in tags)
    any_src = rv["peer"] == ANY_SOURCE
    any_tag = rv["tag"] == ANY_TAG
    assert _within(int(any_src.sum()), nmsg, 0.02)
    if laminar:     # an ANY_SOURCE receive is ANY_TAG too
        assert np.all(any_tag[any_src])
        assert _within(int(any_tag.sum()), nmsg, 1 - 0.95 * 0.98)
    else:
        assert _within(int(any_tag.sum()), nmsg, 0.05)
        assert np.any(any_src & ~any_tag)
    # exact receives of a stream come before its wildcard ones
    for g in range(p.nstreams):
        o = p.ops[p.stream_op_lo[g]: p.stream_op_lo[g + 1]]
        r = o[o["kind"] == IRECV]
        level = (r["tag"] == ANY_TAG).astype(int) + 2 * (r["peer"] == ANY_SOURCE).astype(int)
        assert np.all(np.diff(level) >= 0), f"stream {g}: a wildcard receive before an exact one"
        assert int(o[-1]["kind"]) == WAITALL and int(o[-1]["req_n"]) == len(o) - 1


# ---------------------------------------------------------------------------
# 3-D halo
# ---------------------------------------------------------------------------
@pytest.mark.parametrize("sub", [16, 256])
def test_halo_faces_and_neighbours(sub):
    steps = 2
    p = gen.halo3d(sub=sub, steps=steps, init=False)
    plane = sub * sub
    faces = {}
    for r in range(8):
        ops = p.ops[p.stream_op_lo[r]: p.stream_op_lo[r + 1]]
        assert len(ops) == 13 * steps
        x, y, z = r & 1, (r >> 1) & 1, (r >> 2) & 1
        for s in range(steps):
            o = ops[13 * s: 13 * s + 13]
            assert list(o["kind"][:6]) == [ISEND] * 6 and list(o["kind"][6:12]) == [IRECV] * 6
            assert int(o[12]["kind"]) == WAITALL and int(o[12]["req_n"]) == 12
            for f in range(6):
                snd, rcv = o[f], o[6 + f]
                assert int(snd["tag"]) == f and int(rcv["tag"]) == f ^ 1
                nb = [x, y, z]
                nb[f // 2] += 1 if f % 2 else -1
                dest = (nb[0] % 2) | ((nb[1] % 2) << 1) | ((nb[2] % 2) << 2)
                assert int(snd["peer"]) == dest and int(rcv["peer"]) == dest
                assert type_size(p.types, int(snd["type"])) * int(snd["count"]) == 4 * plane
                assert int(rcv["type"]) == T_FLOAT and int(rcv["count"]) == plane
                t = p.types[int(snd["type"])]
                faces[f] = (int(t["kind"]), int(t["vcount"]), int(t["blocklen"]), int(t["stride"]),
                            int(snd["off"]))
    last = sub - 1
    assert faces[0] == (1, plane, 1, sub, 0) and faces[1] == (1, plane, 1, sub, 4 * last)
    assert faces[2] == (1, sub, sub, plane, 0) and faces[3] == (1, sub, sub, plane, 4 * sub * last)
    assert faces[4][0] == 0 and faces[4][4] == 0 and faces[5][4] == 4 * plane * last
    assert p.meta["payload_bytes"] == steps * 8 * 6 * 4 * plane


# ---------------------------------------------------------------------------
# allreduce inputs
# ---------------------------------------------------------------------------
def test_allreduce_input_distributions():
    n = 1 << 16
    p = gen.allreduce_suite(nranks=4, sizes=(n,), dtypes=(T_INT64, T_FLOAT, T_INT32))
    inst = p.meta["instances"]
    assert [(i["dtype"], i["mode"]) for i in inst] == [
        (T_INT64, MODE_FIXED), (T_FLOAT, MODE_FIXED), (T_FLOAT, MODE_TREE), (T_INT32, MODE_FIXED)]
    assert int(np.count_nonzero(p.ops["kind"] == ALLREDUCE)) == 4 * len(inst)
    N = 4 * n
    v = np.concatenate([p.buf_init[b].view(np.int64) for b in inst[0]["send"]]).astype(np.float64) / 2.0 ** 40
    assert abs(v.mean()) < 5 / math.sqrt(N) and abs(v.std() - 1) < 5 / math.sqrt(2 * N)
    f = np.concatenate([p.buf_init[b].view(np.float32) for b in inst[1]["send"]]).astype(np.float64)
    assert abs(f.mean()) < 5 / math.sqrt(N) and abs(f.std() - 1) < 5 / math.sqrt(2 * N)
    w = np.concatenate([p.buf_init[b].view(np.int32) for b in inst[3]["send"]]).astype(np.float64)
    assert w.min() < -0.99 * 2.0 ** 31 and w.max() > 0.99 * 2.0 ** 31
    assert abs(w.mean()) < 5 * (2.0 ** 32 / math.sqrt(12)) / math.sqrt(N)
    # every rank draws its own values
    assert not np.array_equal(p.buf_init[inst[1]["send"][0]], p.buf_init[inst[1]["send"][1]])


# ---------------------------------------------------------------------------
# serving
# ---------------------------------------------------------------------------
def test_serving_schedule_recipe():
    T, requests, lo, hi, s = 32, 64000, 6, 14, 1.2
    sc = gen.serving_schedule(nthreads=T, requests=requests, min_log2=lo, max_log2=hi, zipf_s=s)
    per = requests // T
    M, nar = sc["messages"], sc["instances"]
    assert nar == round(0.3 * per) and M == (per - nar) * T // 2
    # Zipf(s) over the power-of-two sizes 2^lo..2^hi, rank 1 = 2^lo
    mb = np.asarray(sc["mbytes"], np.int64)
    assert np.all(mb & (mb - 1) == 0)
    k = np.log2(mb).astype(np.int64) - lo
    pmf = 1.0 / np.arange(1, hi - lo + 2) ** s
    pmf /= pmf.sum()
    counts = np.bincount(k, minlength=hi - lo + 1)
    assert len(counts) == hi - lo + 1
    assert all(_within(int(c), M, float(q)) for c, q in zip(counts, pmf))
    calls, call_lo = sc["calls"], sc["call_lo"]
    seen_tags = {}
    for t in range(T):
        c = calls[int(call_lo[t]): int(call_lo[t + 1])]
        kinds = [int(x) for x in c["kind"]]
        # every thread makes its share of calls: sends + receives + allreduces
        assert sum(1 for x in kinds if x != gen.SERVE_WAITALL) > 0
        assert kinds.count(gen.SERVE_ALLREDUCE) == nar
        # an epoch's p2p calls end with a waitall before the epoch's allreduce
        for i, x in enumerate(kinds):
            if x == gen.SERVE_ALLREDUCE and i > 0:
                assert kinds[i - 1] in (gen.SERVE_WAITALL, gen.SERVE_ALLREDUCE)
        for x in c[c["kind"] == gen.SERVE_SEND]:
            assert int(x["peer"]) != t
            seen_tags.setdefault((t, int(x["peer"])), []).append((int(x["item"]), int(x["tag"])))
    total = sum(len(v) for v in seen_tags.values())
    assert total == M
    for v in seen_tags.values():         # the tag counts a pair's messages in item order
        assert [tag for _, tag in sorted(v)] == list(range(len(v)))
    nsr = int(np.count_nonzero(calls["kind"] == gen.SERVE_SEND))
    nrv = int(np.count_nonzero(calls["kind"] == gen.SERVE_RECV))
    nal = int(np.count_nonzero(calls["kind"] == gen.SERVE_ALLREDUCE))
    assert nsr == nrv == M and nal == T * nar
    assert abs(nal / (nal + nsr + nrv) - 0.3) < 0.01
