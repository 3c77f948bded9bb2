"""GB300-native walk-on-boundary (WoB) estimator."""
