"""The accuracy contract of gmrf_sample, shared by the GPU parity tests: a
vector returned with status OK meets the tolerance (its error against the
oracle is within the bound the test states), and a vector the library could
not bring there is returned as NOT_CONVERGED with an error estimate that
covers the error it has."""

OK = 0
NOT_CONVERGED = -3


def assert_honest(info, err, bound, slack=0.0):
    """info: the vector's SampleInfo; err: its error against the oracle;
    bound: what status OK promises for this case; slack: error the test
    states to lie outside the iteration's estimate (e.g. the rounding of a
    final map after the iteration)."""
    if info.status == OK:
        assert err <= bound, (err, bound, info)
    else:
        assert info.status == NOT_CONVERGED, info
        assert info.err_est + slack >= err, (err, info)
