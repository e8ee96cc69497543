"""Host model of the warp-specialised tile pass's barrier protocol
(k_tile_impl.cuh, tile_pass_ws_kernel), checked under random interleavings
with out-of-order completion of the tensor loads.

The model follows the kernel: a producer walks the tiles in order, stores
tile j - NB from buffer j % NB once that buffer's empty barrier completed the
phase of tile j - NB, then loads tile j into it; consumer group g takes the
tiles g, g + 2, ..., waits for the tile's load with try_wait.parity, runs,
and arrives on the buffer's empty barrier.  An mbarrier is modelled by its
count of completed phases; try_wait.parity(P) succeeds when that count's
parity differs from P.  With a load completing on the barrier of its
(buffer, group) pair and parity (k / lcm(NB, 2)) & 1 (the kernel's form) no
consumer ever starts a tile whose data has not landed and no load lands in a
buffer in use.  The form with one barrier per buffer and parity (k / NB) & 1
fails under out-of-order loads, which is what the pair barriers fix."""
import random


def simulate(nb, n_tiles, pair_barriers, seed):
    rnd = random.Random(seed)
    full = [0] * 8
    empty = [0] * nb
    landed = [None] * nb
    inflight = []
    period = (2 * nb if nb % 2 else nb) if pair_barriers else nb

    def fidx(b, g):
        return 2 * b + g if pair_barriers else b

    j_next = 0
    cons = [{"k": g, "busy": 0, "working": False} for g in (0, 1)]
    in_use = {}
    stored = []
    errors = []
    for _ in range(100000):
        acts = []
        if j_next < n_tiles + nb:
            acts.append("producer")
        if inflight:
            acts.append("land")
        acts += [("consumer", g) for g in (0, 1) if cons[g]["k"] < n_tiles]
        if not acts:
            break
        a = rnd.choice(acts)
        if a == "producer":
            j, b = j_next, j_next % nb
            if j >= nb:
                u = (j - nb) // nb
                if (empty[b] & 1) == (u & 1):   # the release of tile j - nb has not completed
                    continue
                stored.append(j - nb)
            if j < n_tiles:
                if b in in_use:
                    errors.append(("load into a buffer in use", j, b))
                inflight.append((j, b, fidx(b, j & 1)))
            j_next += 1
        elif a == "land":
            j, b, f = inflight.pop(rnd.randrange(len(inflight)))   # any order
            landed[b] = j
            full[f] += 1
        else:
            g = a[1]
            c = cons[g]
            k, b = c["k"], c["k"] % nb
            if not c["working"]:
                if (full[fidx(b, g)] & 1) != ((k // period) & 1):   # try_wait.parity succeeds
                    if landed[b] != k:
                        errors.append(("consumer started before its tile landed", g, k, landed[b]))
                    in_use[b] = k
                    c["working"], c["busy"] = True, rnd.randint(0, 3)
            elif c["busy"]:
                c["busy"] -= 1
            else:
                in_use.pop(b, None)
                empty[b] += 1
                c["k"] += 2
                c["working"] = False
    if sorted(stored) != list(range(n_tiles)):
        errors.append(("not every tile was stored", len(stored)))
    return errors


def test_pair_barriers_keep_the_pipeline_exact():
    for nb in (3, 4):
        for seed in range(200):
            assert simulate(nb, 61, True, seed) == [], (nb, seed)


def test_one_barrier_per_buffer_races_with_three_buffers():
    assert any(simulate(3, 60, False, seed) for seed in range(200))
