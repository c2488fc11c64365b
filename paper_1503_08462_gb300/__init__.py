"""GB300-native solve phase of the AMG multilevel-correction eigensolver."""
