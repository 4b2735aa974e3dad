"""A plain restatement of the library's parallel cuckoo placement
(pepsi_params.client_cuckoo = 1), round by round, for the tests: every
unplaced item claims its current candidate bin; the smallest claimant of a
bin takes its first free slot, or evicts the occupant of slot (evictions mod
gamma), which moves on to its next candidate; the other claimants move on to
theirs.  Returns where[u] = bin * gamma + slot, or None after max_rounds."""


def rounds_reference(bins3, gamma, nbins, max_rounds=1000):
    m = len(bins3)
    state, choice = [1] * m, [0] * m
    slot = [-1] * (nbins * gamma)
    load, evictions = [0] * nbins, [0] * nbins
    for _ in range(max_rounds):
        claim = {}
        for u in range(m):
            if state[u] == 1:
                b = bins3[u][choice[u]]
                claim[b] = min(claim.get(b, m), u)
        for b, w in claim.items():
            if load[b] < gamma:
                c = b * gamma + load[b]
                load[b] += 1
            else:
                c = b * gamma + evictions[b] % gamma
                evictions[b] += 1
                v = slot[c]
                state[v], choice[v] = 2, (choice[v] + 1) % 3
            slot[c], state[w] = w, 0
        left = 0
        for u in range(m):
            if state[u] == 1:
                choice[u] = (choice[u] + 1) % 3
                left += 1
            elif state[u] == 2:
                state[u] = 1
                left += 1
        if not left:
            where = [-1] * m
            for c, u in enumerate(slot):
                if u >= 0:
                    where[u] = c
            return where
    return None
