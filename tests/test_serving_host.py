"""Host-side serving logic that needs no GPU."""
def test_serving_batch_size_policy():
    """Batch sizes: powers of two taken down from the queue, capped by
    max_batch and by the per-volume device-time budget (host logic only)."""
    from paper_2402_15641_gb300.serving import batch_size
    assert batch_size(1, 16, None, 0.01) == 1
    assert batch_size(3, 16, None, 0.01) == 2
    assert batch_size(16, 16, None, 0.01) == 16
    assert batch_size(40, 16, None, 0.01) == 16
    assert batch_size(40, 16, 0.001, 0.01) == 8     # 10 volumes fit, rounded down to 8
    assert batch_size(40, 16, 0.004, 0.01) == 2
    assert batch_size(40, 16, 0.05, 0.01) == 1      # one volume exceeds the budget alone
    assert batch_size(5, 1, None, 0.01) == 1        # unbatched server
