"""GB300-native open-boundary RPY mobility: M(X)[F;T] and sqrt(M) W."""
