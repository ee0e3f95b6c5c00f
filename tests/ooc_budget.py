"""Device budgets for out-of-core test contexts, by the rule VR_OPT_DEVICE_BUDGET
documents: the direct march takes one block of (bx+1)(by+1)(bz+1) floats per cache
slot; the texture march takes its layered copies per slot (three, two along x and z, or one along z)
plus a staging area of max(min(64 MiB of blocks, slots / 8), ring half) blocks,
sized for the slots the budget would hold without it."""


def block_bytes(brick):
    return (brick[0] + 1) * (brick[1] + 1) * (brick[2] + 1) * 4


def stage_blocks(slots, brick):
    group = max(1, (64 << 20) // block_bytes(brick))
    eighth = max(1, slots // 8)
    half = max(1, min(slots // 8, 32))
    return max(min(group, eighth), half)


def slots_of(budget, brick, march, n_bricks):
    """Cache slots that a budget gives (march 0: direct, 1: three copies, 3: one,
    4: two)."""
    blocks = budget // block_bytes(brick)
    if march == 0:
        return min(n_bricks, blocks)
    copies = {1: 3, 3: 1, 4: 2}[march]
    return min(n_bricks, (blocks - stage_blocks(blocks // copies, brick)) // copies)


def budget_for(slots, brick, march, n_bricks=1 << 30):
    """The smallest budget (bytes) whose cache has exactly `slots` slots."""
    b = block_bytes(brick)
    blocks = slots
    while slots_of(blocks * b, brick, march, n_bricks) < slots:
        blocks += 1
    assert slots_of(blocks * b, brick, march, n_bricks) == slots
    return blocks * b
